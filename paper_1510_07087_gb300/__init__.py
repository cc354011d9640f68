"""GB300 (sm_103a) directional H^2-matrix compression.

The compute path is the C-ABI CUDA library `libdh2.so` (include/dh2.h); this
package is its Python binding (argument marshalling only).
"""
from ._binding import (  # noqa: F401
    DH2_C64, DH2_C128, MODE_FP32, MODE_FP64, MODE_MIXED_BF16X3, SIDE_COL, SIDE_ROW,
    KC_CLASSIFY, KC_COLW, KC_COUNT, KC_EXPAND, KC_GRAM_SCALES, KC_LEAF_JACOBI, KC_LEAF_R_TC, KC_LEAF_FACTOR, KC_LEAF_GRAM, KC_LEAF_R, KC_LEVEL_FACTOR, KC_LEVEL_R, KC_NORMS,
    KC_PROJECT,
    DH2Error, Plan, ERR_FRO_BLOCKWISE, ERR_FRO_CLOSED, ERR_SPECTRAL, Matrix, Tree,
    autotune, set_tuning, tuning,
    dh2_compress, dh2_compress_batched, dh2_compress_host, dh2_compress_kernel, dh2_compress_kernel_dlp, dh2_debug_fail_alloc, dh2_error, dh2_matvec_adjoint, dh2_matvec, dh2_matvec_noalloc, dh2_tree_build, dh2_version, exported_symbols,
)
