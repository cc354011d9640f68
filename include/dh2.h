/*
 * dh2.h - C ABI of the GB300 directional H^2-matrix compression library.
 *
 * The library approximates a dense complex matrix G in C^{I x I} by a
 * directional H^2 (DH^2) matrix: orthonormal directional row and column
 * cluster bases V, W given by leaf matrices and transfer matrices E
 * (Def. "Directional cluster basis", Eq. nested), coupling matrices
 * S_b = V_tc^* G|_{t x s} W_sc for admissible leaves b = (t, s) with block
 * direction c = c_b (Def. "Directional H^2-matrix", Section 6), and the
 * nearfield blocks G|_b of the inadmissible leaves.  The bases are built
 * bottom-up by the compression procedure of Section 6 (procedure basis()
 * of the figure "Construction of an orthogonal directional cluster basis")
 * applied to G for V and to G^* for W.
 *
 * Conventions for every entry point:
 *  - Return value: a dh2_status; no exception crosses the ABI.  On failure an
 *    output handle is set to NULL and nothing is leaked.
 *  - Index order: every device vector and matrix is in the tree's PERMUTED
 *    order, in which each cluster is a contiguous index range; dh2_tree_perm
 *    gives the map back to the caller's order.
 *  - Complex data are interleaved (re, im) pairs: DH2_C64 = 2 x float,
 *    DH2_C128 = 2 x double.  Matrices are column-major with a leading
 *    dimension `ld` >= n (in elements).
 *  - Streams: calls that take a cudaStream_t (passed as void*) enqueue their
 *    GPU work on it; dh2_compress synchronises that stream once at its end to
 *    read the device status word (NULL = the legacy default stream).
 *  - Ownership: the caller owns G, x, y and the points; the library owns
 *    everything behind a handle and frees it in dh2_*_free.  In nearfield VIEW
 *    mode the matrix handle keeps a pointer to G, which must outlive it.
 *  - Host-only calls (tree build, tree queries) never touch a GPU.
 */
#ifndef DH2_H
#define DH2_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dh2_tree dh2_tree;     /* cluster tree, directions, block tree, work lists */
typedef struct dh2_matrix dh2_matrix; /* device-resident DH^2 representation             */

typedef enum {
  DH2_OK = 0,
  DH2_EINVAL = 1,       /* bad argument (null pointer, size, parameter range)       */
  DH2_ENOMEM = 2,       /* host or device allocation failed                         */
  DH2_ECUDA = 3,        /* a CUDA runtime call failed                               */
  DH2_ETIMEOUT = 4,     /* a bounded device-side wait ran out                        */
  DH2_ENOCONV = 5,      /* a Jacobi SVD hit its sweep cap, or met non-finite values  */
  DH2_EUNSUPPORTED = 6  /* size beyond a compiled limit (e.g. rows of a factor)      */
} dh2_status;

typedef enum { DH2_C64 = 0, DH2_C128 = 1 } dh2_dtype;

/* Arithmetic of the compression.
 *  FP64: complex128 input and FP64 everywhere (the plain form).
 *  FP32: complex64 input, FP32 factorisations on the non-squared factors
 *        (streamed Householder LQ), FP64 tail sums for the rank decisions.
 *  MIXED_BF16X3: complex64 input; the leaf step of Section 6 reduces each
 *        leaf matrix G^omega_tc to its Gram matrix on the tensor cores
 *        (tcgen05, bf16 operands, FP32 accumulation in tensor memory) from
 *        three 8-bit fixed-point slices per entry, scaled per row, with every
 *        accumulation exact, so the Gram matrix is that of a matrix within
 *        2^-23 of each row's largest entry of G^omega_tc, to ~48 bits; the
 *        rank-revealing step is a pivoted Cholesky of it in double-float
 *        arithmetic, followed by the same FP32 Jacobi, FP64 tail sums, R, level
 *        steps and projection as FP32.  Leaves of at most 64 rows, dense G
 *        only (not the matrix-free entry points).  For eps >= 1e-5: below
 *        that the squared singular values are no longer resolved to the tail
 *        sums' precision, and the call (unless keep_gram is set) runs the
 *        FP32 mode's leaf step instead; its result is then the FP32 mode's. */
typedef enum { DH2_MODE_FP64 = 0, DH2_MODE_FP32 = 1, DH2_MODE_MIXED_BF16X3 = 2 } dh2_mode;

/* Tree parameters (Section 3; Section 7 for the paper's values).
 *  leaf_size : a cluster with more indices is bisected (Def. 1).
 *  kappa     : wave number of Eq. (helmholtz) and Eq. (adm_parabolic).
 *  eta1      : direction parameter of Eq. (adm_directional): D_l covers the
 *              sphere with radius eta1 / (kappa * delta_l).
 *  eta2      : parameter of Eqs. (adm_parabolic) and (adm_standard).
 *  dir_rule  : 0 = cube-surface directions on every level, 1 = {0} on levels
 *              with kappa * delta_l <= eta1 (Def. 3 allows c = 0). */
typedef struct {
  int32_t leaf_size;
  int32_t dir_rule;
  double kappa;
  double eta1;
  double eta2;
} dh2_tree_params;

/* Compression parameters (Remark "Error control").
 *  eps       : requested accuracy.
 *  zeta      : level factor of eps_r = eps_hat * zeta^level(r), zeta < 1/sqrt 2.
 *  err_mode  : 0 = eps_hat = eps*sqrt(1-2 zeta^2)/sqrt 2, which bounds
 *              |G - G~|_F <= eps |G|_F; 1 = eps_hat = eps.
 *  mode      : dh2_mode; must match the dtype of G (FP64 <-> C128, FP32 and
 *              MIXED_BF16X3 <-> C64).
 *  nearfield : 0 = copy the inadmissible blocks into the matrix handle,
 *              1 = keep a view of G.
 *  max_sweeps: cap on Jacobi sweeps per factor (0 = default 30).
 *  rank_override: NULL, or per side (0 row, 1 column) a host array of one
 *              rank per used pair (dh2_tree_pairs order), read during the
 *              call; an entry >= 0 replaces the truncation rule for that pair
 *              (clamped to the singular values the factorisation resolves and
 *              to the rank capacity), an entry < 0 keeps the rule.  With the
 *              ranks of another implementation (an oracle) both compute the
 *              same approximation.  Either side's pointer may be NULL.
 *  spin_limit: polls of a bounded device-side wait (the mixed modes' wait
 *              for tensor-core batches) before it gives up, sets the timeout
 *              status and returns DH2_ETIMEOUT; 0 = default (about a second).
 *  keep_gram : mixed modes, instrumentation: keep the leaf Gram matrices in
 *              the matrix handle for dh2_matrix_leaf_gram (0 = free them).  */
typedef struct {
  double eps;
  double zeta;
  int32_t err_mode;
  int32_t mode;
  int32_t nearfield;
  int32_t max_sweeps;
  const int32_t* rank_override[2];
  int64_t spin_limit;
  int32_t keep_gram;
  int32_t reserved;
} dh2_compress_params;

typedef struct {
  int64_t n;
  int32_t depth;           /* p_I of Def. 1                                  */
  int32_t nclusters;
  int64_t nblocks;         /* leaves of the block tree                        */
  int64_t nadmissible;     /* admissible leaves                               */
  double adm_fraction;     /* admissible entries / n^2                        */
  int64_t npairs[2];       /* used (t, c) pairs, [0] row side, [1] column side */
  int64_t nleafpairs[2];
  int64_t ncolumns[2];     /* sum over pairs of #F_tc                          */
  int64_t nleafcolumns[2]; /* sum over leaf pairs of #F_tc                     */
  int32_t max_leaf;        /* largest leaf cluster                            */
  int32_t ndirs_max;       /* largest |D_l|                                    */
} dh2_tree_stats;

/* ---------------------------------------------------------------- tree (host) */

/* Build the cluster tree (Def. 1, bisection of tight bounding boxes at the
 * midpoint of the longest side), the direction families D_l and son maps
 * sd_l (Def. 3, Section 3), the block tree (Def. 2 with Eqs. adm_parabolic and
 * adm_standard), the block directions c_b and, for both sides, the used
 * (cluster, direction) pairs with their column sets F_tc (Section 6).
 * pts_xyz: host, n x 3 row-major doubles, read only during the call. */
dh2_status dh2_tree_build(const double* pts_xyz, int64_t n, const dh2_tree_params* params,
                          dh2_tree** out);
void dh2_tree_free(dh2_tree* tree);
dh2_status dh2_tree_stats_get(const dh2_tree* tree, dh2_tree_stats* out);
/* perm[i] = caller index of permuted index i (host, n entries). */
dh2_status dh2_tree_perm(const dh2_tree* tree, int64_t* perm);
/* Per-cluster arrays (host, nclusters entries each; lo/hi 3 per cluster;
 * son0/son1 = -1 for leaves).  Any pointer may be NULL. */
dh2_status dh2_tree_clusters(const dh2_tree* tree, int32_t* start, int32_t* size, int32_t* level,
                             int32_t* parent, int32_t* son0, int32_t* son1, double* lo, double* hi);
/* Number of directions on a level, then the directions (3 doubles each) and
 * the son map into level+1 (-1 on the deepest level).  Either pointer may be NULL. */
dh2_status dh2_tree_ndirs(const dh2_tree* tree, int32_t level, int32_t* ndirs);
dh2_status dh2_tree_directions(const dh2_tree* tree, int32_t level, double* dirs, int32_t* sd);
/* Leaves of the block tree in construction order (host, nblocks entries each):
 * row cluster, column cluster, admissible flag, block direction (-1 if not admissible). */
dh2_status dh2_tree_blocks(const dh2_tree* tree, int32_t* t, int32_t* s, int32_t* adm, int32_t* cb);
/* Used pairs of one side (0 row, 1 column): cluster, direction, #F_tc columns,
 * leaf flag; and the blocks of F_tc in the library's column order as CSR
 * (offsets: npairs+1 entries; block ids: offsets[npairs] entries).  A NULL
 * `block_ids` with non-NULL `offsets` returns only the offsets. */
dh2_status dh2_tree_pairs(const dh2_tree* tree, int32_t side, int32_t* cluster, int32_t* dir,
                          int64_t* ncols, int32_t* is_leaf);
dh2_status dh2_tree_pair_blocks(const dh2_tree* tree, int32_t side, int64_t* offsets, int32_t* block_ids);
/* Column panels of dh2_compress_host (built on first use and kept in the tree):
 * *npanels; col[0..npanels] the panel boundaries in the permuted order (may be
 * NULL); row_panel[p] for each row-basis pair p the panel after whose arrival
 * its leaf factor runs, -1 for a non-leaf pair (may be NULL). */
dh2_status dh2_tree_panels(const dh2_tree* tree, int32_t* npanels, int64_t* col, int32_t* row_panel);

/* ---------------------------------------------------------------- compression (GPU) */

/* Compress G (device, n x n column-major, permuted order, leading dimension
 * ld) into a DH^2 matrix.  Realises procedure basis() of Section 6 for the row
 * basis and for the column basis (the same procedure on G^*), with the
 * weighted error control of Remark "Error control" (omega_b = |G_b|_F *
 * zeta^-level(t)), followed by the projection S_b = V_tc^* G_b W_sc.
 * Errors: DH2_EINVAL for bad sizes/params or a dtype/mode mismatch,
 * DH2_ENOCONV / DH2_EUNSUPPORTED from the device status word, DH2_ECUDA. */
dh2_status dh2_compress(const dh2_tree* tree, const void* G, dh2_dtype dtype, int64_t ld,
                        const dh2_compress_params* params, void* stream, dh2_matrix** out);

/* The same compression of a G held in HOST memory (n x n column-major,
 * permuted order, leading dimension ld >= n; page-locked memory gives the
 * full copy rate, pageable memory is accepted).  The library copies G into a
 * device buffer owned by the tree (n*n elements of the dtype, allocated on
 * the first call and kept until dh2_tree_free; a larger dtype reallocates it
 * and synchronises the device).  The copy runs in column panels made of whole
 * clusters of the shallowest level that holds an admissible block, on a
 * second stream: each panel's block norms, nearfield copies and column-basis
 * leaf factors (which read only that panel's columns of G, Section 6 applied
 * to G^*), and the row-basis leaf factors whose columns lie in the panels
 * copied so far, run while the next panel is copied.  Copy mode only
 * (params->nearfield == 0): the buffer is reused by the next call on the same
 * tree, so calls on one tree must be ordered (same stream, or synchronised).
 * The call returns when the compression is complete, so G_host may be freed
 * after it; the matrix keeps no reference to G (dh2_error needs the
 * reference passed explicitly).  Errors as dh2_compress;
 * DH2_EINVAL also for view mode, DH2_ENOMEM if the buffer cannot be allocated. */
dh2_status dh2_compress_host(const dh2_tree* tree, const void* G_host, dh2_dtype dtype, int64_t ld,
                             const dh2_compress_params* params, void* stream, dh2_matrix** out);
/* Compress nprob independent matrices (each with its own tree, size and
 * leading dimension; same dtype and parameters) in one schedule: block norms,
 * leaf factorisations and every level of non-leaf steps are each one launch
 * over all problems.  out: array of nprob handles (all NULL on failure).
 * nprob <= 64; each problem as for dh2_compress. */
dh2_status dh2_compress_batched(int32_t nprob, const dh2_tree* const* trees, const void* const* G,
                                const int64_t* ld, dh2_dtype dtype, const dh2_compress_params* params,
                                void* stream, dh2_matrix** out);

/* Matrix-free compression of the Helmholtz collocation matrix
 * G_ij = exp(i kappa |x_i - x_j|) / (4 pi |x_i - x_j|) (Eq. helmholtz), with
 * `diag` on the diagonal: every entry the compression reads (block norms,
 * leaf factors, R, nearfield copy) is generated in the kernels from the
 * points, so no dense G is needed.  pts_xyz: host, n x 3 row-major doubles in
 * the caller's order (the array given to dh2_tree_build), copied during the
 * call.  params->mode selects FP32 (complex64 entries: distances and phase
 * reduction in FP64, sin/cos of the reduced phase in FP32) or FP64.  The
 * nearfield is always copied (params->nearfield must be 0).  dh2_error on the
 * result accepts G_ref = NULL: the reference is then generated in FP64. */
dh2_status dh2_compress_kernel(const dh2_tree* tree, const double* pts_xyz, double kappa, double diag,
                               const dh2_compress_params* params, void* stream, dh2_matrix** out);

/* Matrix-free compression of the double-layer collocation matrix of the
 * paper's second experiment (Section 7, "DLP matrix"):
 * G_ij = (1 - i kappa r) exp(i kappa r) / (4 pi r^3) <x_i - x_j, n(x_j)>,
 * r = |x_i - x_j|, and G_ii = 1/2 (the identity standing in for the mass
 * matrix of 1/2 M + G_dlp).  normals_xyz: host, n x 3 row-major unit normals
 * in the caller's order, copied during the call.  Otherwise as
 * dh2_compress_kernel; dh2_error with G_ref = NULL generates this matrix. */
dh2_status dh2_compress_kernel_dlp(const dh2_tree* tree, const double* pts_xyz, const double* normals_xyz,
                                   double kappa, const dh2_compress_params* params, void* stream,
                                   dh2_matrix** out);
/* ---------------------------------------------------------------- captured schedule
 * The compression of one problem, or of nprob independent problems as by
 * dh2_compress_batched, prepared once and captured into a CUDA graph: the
 * representation(s) are allocated, the launch lists and argument blocks
 * uploaded and the kernel sequence (block norms and nearfield, leaf factors
 * and R, the level steps with their capacity launches, expansion, projection)
 * recorded without running it.  dh2_plan_run replays the whole sequence with
 * one graph launch on new matrices of the same shapes and leading dimensions;
 * no allocation, upload of a launch list or host synchronisation happens in
 * it.  The representation is the same as dh2_compress / dh2_compress_batched
 * would produce for those matrices.  G, ld, dtype, params: as for
 * dh2_compress_batched (device matrices only; G gives the first inputs).
 * The plan owns its matrices (dh2_plan_matrix lends them; they stay valid
 * until dh2_plan_free and are rewritten by every run).  Errors: EINVAL,
 * ENOMEM, ECUDA, EUNSUPPORTED (a class beyond the device's shared memory; the
 * debug and profile builds, which synchronise inside the schedule).  A run's
 * device status (timeout, non-convergence, non-finite input) is returned by
 * dh2_plan_wait, which synchronises the stream.  Runs on one plan are
 * stream-ordered: do not run one plan on two streams at once.  The paper has
 * no counterpart (scheduling). */
typedef struct dh2_plan dh2_plan;
dh2_status dh2_plan_create(int32_t nprob, const dh2_tree* const* trees, const void* const* G, const int64_t* ld,
                           dh2_dtype dtype, const dh2_compress_params* params, void* stream, dh2_plan** out);
/* G: nprob device matrices, or NULL for those of the previous run. */
dh2_status dh2_plan_run(dh2_plan* P, const void* const* G, void* stream);
dh2_status dh2_plan_wait(dh2_plan* P, void* stream);
dh2_status dh2_plan_matrix(const dh2_plan* P, int32_t i, dh2_matrix** M);
void dh2_plan_free(dh2_plan* P);

/* ---------------------------------------------------------------- autotuning
 * Launch choices of the compression that change its time, not its steps
 * (Section 6's procedure is the same under every choice).  One table per
 * process, read by each later compression when it prepares its launches (a
 * plan keeps the choices it was captured with).
 *  jacobi_tpp[c]   : most threads per column pair of a Jacobi round, factor
 *                    class c (rows <= 32, <= 40, <= 48, <= 64, more): 4, 8,
 *                    16 or 32 (default 32).  Changes the summation order of
 *                    the rotation sums, so results move by rounding only.
 *  jacobi_narrow[c]: mixed mode, leaf classes 0..3: threads per CTA of the
 *                    Jacobi launch, 0 = 4 x rows, 1 = about 2 x rows
 *                    (default), 2 = about 1 x rows (a multiple of 32), at the
 *                    same threads per SM.  Changes the rounding as above.
 *  rq_ctas_per_sm  : resident CTAs per SM of the persistent leaf R kernel
 *                    of the FP32 pipes, 1..4 within its occupancy limit, 0 =
 *                    that limit (default).  Changes no result.
 *  rq_tensor       : mixed mode: 1 = the leaf R on the tensor cores (bf16
 *                    slices, FP32 accumulation), 0 = on the FP32 pipes
 *                    (default, measured faster).  The two agree to FP32
 *                    rounding.
 *  level_seg_cols  : non-leaf pairs with more than 2 x level_seg_cols
 *                    columns are factored in column segments of that width
 *                    (each segment's LQ factor L_i by its own CTA, then the
 *                    pair's factor from [L_1 ... L_S], which has the same
 *                    singular values and left singular vectors); 0 = never
 *                    split, else a multiple of 64 from 256 to 8192 (default
 *                    1024).  Changes the rounding only.
 * dh2_tuning_set returns DH2_EINVAL (table unchanged) for a value outside
 * these sets. */
typedef struct {
  int32_t jacobi_tpp[5];
  int32_t jacobi_narrow[4];
  int32_t rq_ctas_per_sm;
  int32_t rq_tensor;
  int32_t level_seg_cols;
} dh2_tuning;
dh2_status dh2_tuning_get(dh2_tuning* out);
dh2_status dh2_tuning_set(const dh2_tuning* tuning);
/* One timed candidate of dh2_autotune: knob 0 = rq_ctas_per_sm, 1 =
 * jacobi_narrow[cls], 2 = jacobi_tpp[cls], 3 = rq_tensor, 4 = level_seg_cols;
 * ms = median device time of the phase the knob acts on (leaf R, level
 * steps, or leaf factors) over the repetitions. */
typedef struct {
  int32_t knob;
  int32_t cls;
  int32_t value;
  float ms;
} dh2_tune_record;
/* Autotune the table on one problem: compresses (tree, G) with `params`
 * under each candidate of each knob in turn (coordinate descent: in the
 * mixed mode the R kernel, then the R grid, the level steps' segment width
 * (if a non-leaf pair has more than 1024 columns), then per factor class the
 * Jacobi launch width and the threads per column pair; a
 * class with no pairs in the problem is skipped), `reps` calls per candidate
 * (1..15), keeps the fastest value of each knob, installs the result and
 * returns it in `out`.  records: NULL, or room for `cap` records, of which
 * *nrec are written (every candidate timed, in order; NULL nrec allowed when
 * records is NULL).  The matrices it makes are freed before it returns.
 * Errors: those of dh2_compress (the table is then left as it was), EINVAL
 * for reps outside 1..15. */
dh2_status dh2_autotune(const dh2_tree* tree, const void* G, dh2_dtype dtype, int64_t ld,
                        const dh2_compress_params* params, void* stream, int32_t reps, dh2_tuning* out,
                        dh2_tune_record* records, int32_t cap, int32_t* nrec);

void dh2_matrix_free(dh2_matrix* M);

/* y = G~ x for the compressed matrix (Section 4: forward transformation,
 * coupling, backward transformation, plus the nearfield).  x, y: device,
 * n x nrhs column-major (leading dimension n), permuted order, dtype of the
 * matrix.  y is overwritten.  Preconditions the library cannot check (it
 * receives plain pointers): x and y are allocations on the matrix's device
 * holding at least n * nrhs elements of the matrix's complex type (complex64
 * for DH2_MODE_FP32, complex128 for DH2_MODE_FP64); a shorter or wrongly typed
 * buffer is read or written out of bounds.  The Python binding checks dtype,
 * device, row count and shape before the call. */
dh2_status dh2_matvec(const dh2_matrix* M, const void* x, void* y, int32_t nrhs, void* stream);

/* Same product as dh2_matvec, for callers that must not allocate device
 * memory during the call -- for example a solver that reserves all of its
 * memory once at start-up and may not grow past that budget, or a component
 * running next to an allocator that others own.  This entry point has no
 * counterpart in the paper; it exists for those callers only.
 * It performs no cudaMalloc/cudaFree and calls no allocating library routine:
 * the per-pair coefficient vectors live in one fixed, library-owned device
 * array of 8 MiB, which every GPU that loads the library holds until the
 * process exits.  Requirements and behaviour:
 *  - the coefficient vectors need sum over pairs of k_cap(t,c) * nrhs complex
 *    entries for each basis; if that exceeds 8 MiB the call returns
 *    DH2_EUNSUPPORTED and does nothing (use dh2_matvec, or fewer columns);
 *  - the device of M must be the current device (else DH2_EINVAL); the first
 *    call on a device looks the array's device address up once (a CUDA
 *    runtime query, not an allocation), so make that first call before any
 *    stream capture;
 *  - every call uses the same array and it keeps the last call's contents;
 *    each call writes every coefficient before reading it, but calls whose
 *    work overlaps on the GPU (different streams, or different threads without
 *    ordering) race on the array: order them on one stream;
 *  - the array's device address is looked up once per device and cached for
 *    the life of the process: after cudaDeviceReset (or any other teardown of
 *    the device's primary context) the cached address is stale, so do not
 *    call this entry point again in such a process.
 * x, y: as for dh2_matvec; y is overwritten. */
dh2_status dh2_matvec_noalloc(const dh2_matrix* M, const void* x, void* y, int32_t nrhs, void* stream);

/* y = G~^* x, the adjoint of dh2_matvec's product: the transformations of
 * Section 4 with the roles of the row and column bases exchanged (forward on
 * V, coupling with S_b^*, backward on W) plus G_b^* on the nearfield.
 * Arguments and preconditions as dh2_matvec. */
dh2_status dh2_matvec_adjoint(const dh2_matrix* M, const void* x, void* y, int32_t nrhs, void* stream);

/* Error measures of dh2_error. */
enum {
  DH2_ERR_FRO_BLOCKWISE = 0, /* |G_ref - G~|_F / |G_ref|_F, block by block (FP64 sums)          */
  DH2_ERR_FRO_CLOSED = 1,    /* the same from sum_b |G_b|_F^2 - |S_b|_F^2 over admissible blocks,
                                the squared error of the orthogonal projection (Section 6,
                                Def. "Orthogonality"; exact for orthonormal bases); G_ref is not
                                read (the block norms of the compressed G are used), so the value
                                only means something in FP64 mode: in the complex64 modes the
                                difference is below the rounding of the two norms             */
  DH2_ERR_SPECTRAL = 2       /* |G_ref - G~|_2 / |G_ref|_2 by power iteration (the measure of
                                the paper's experiments, Section 7): products with G_ref, G_ref^*
                                in FP64 and with G~, G~^* (dh2_matvec, dh2_matvec_adjoint), from a
                                fixed seeded start vector, until the estimate changes by less than
                                1e-6 relative or after 60 products                             */
};
/* Relative error of the compressed matrix against G_ref, a device matrix of
 * dtype ref_dtype (n x n column-major, permuted order, leading dimension ld),
 * or NULL for a matrix from dh2_compress_kernel[_dlp] (reference entries
 * generated in FP64), by the measure `which`.  Synchronises the stream. */
dh2_status dh2_error(const dh2_matrix* M, const void* G_ref, dh2_dtype ref_dtype, int64_t ld, int32_t which,
                     void* stream, double* rel_err);

/* Ranks of the used pairs of one side (host, npairs entries; may be NULL when the side has no pair). */
dh2_status dh2_matrix_ranks(const dh2_matrix* M, int32_t side, int32_t* ranks);
/* Singular values resolved individually for one pair (host, up to `cap`
 * doubles, sorted descending); *count receives how many were resolved.  The
 * factorisation stops resolving once the remaining energy is below a small
 * fraction of eps_l^2; dh2_matrix_sigma_rest gives that energy (the sum of
 * the squares of the unresolved singular values, up to rounding). */
dh2_status dh2_matrix_sigma(const dh2_matrix* M, int32_t side, int64_t pair, double* out, int32_t cap,
                            int32_t* count);
dh2_status dh2_matrix_sigma_rest(const dh2_matrix* M, int32_t side, int64_t pair, double* energy);
/* Stored matrix of one pair, copied to the host as complex128: a leaf pair's
 * basis Q_tc (rows = cluster size) or a non-leaf pair's [E_t1c; E_t2c]
 * (rows = k_t1c' + k_t2c').  out: rows x k column-major, ld = rows. */
dh2_status dh2_matrix_pair_basis(const dh2_matrix* M, int32_t side, int64_t pair, double* out,
                                 int64_t cap_elems, int32_t* rows, int32_t* k);
/* Coupling matrix S_b of an admissible block, copied to the host as complex128
 * (k_t x k_s column-major). */
dh2_status dh2_matrix_coupling(const dh2_matrix* M, int64_t block, double* out, int64_t cap_elems,
                               int32_t* kt, int32_t* ks);
/* Weights 1/omega_b of the blocks (Remark "Error control": omega_b =
 * |G_b|_F zeta^-level(t) for an admissible block, 1 for a zero block; entries
 * of inadmissible blocks are unspecified).  invw: host, nblocks doubles. */
dh2_status dh2_matrix_block_weights(const dh2_matrix* M, double* invw);
/* Leaf Gram matrix H = A A^* of one leaf pair from the tensor-core kernel of
 * the mixed modes (A = G^omega_tc of Section 6's leaf step, with the weights
 * above rounded to FP32), for a matrix compressed with keep_gram = 1:
 * copied to the host as complex128 (hi + lo of each double-float entry),
 * m x m column-major with m the cluster size (*m receives it).  out holds
 * at least cap_elems complex entries.  Instrumentation only: DH2_EINVAL if
 * the matrix kept no Gram matrices or the pair is not a leaf. */
dh2_status dh2_matrix_leaf_gram(const dh2_matrix* M, int32_t side, int64_t pair, double* out, int64_t cap_elems,
                                int32_t* m);
/* Storage in stored entries (Def. "DH^2-matrix representation"):
 * parts[0..5] = V leaves, W leaves, E of V, E of W, S, nearfield; *total = sum. */
dh2_status dh2_storage(const dh2_matrix* M, double* total, double* parts);
/* Time of the last dh2_compress per phase in ms measured with CUDA events
 * (ms6: host array of 6 floats): [0] norms+nearfield, [1] leaf factors,
 * [2] leaf R = Q^* A, [3] level steps (factors and R), [4] expansion,
 * [5] projection. */
dh2_status dh2_matrix_phase_ms(const dh2_matrix* M, float* ms6);
/* The leaf-factor phase of the last dh2_compress in the mixed modes with G on
 * the device, split by kernel (ms2: host array of 2 floats, CUDA events around
 * each launch): [0] the tensor-core Gram launches, [1] the pivoted Cholesky,
 * Jacobi and truncation launches.  Both 0 in the other modes and for host
 * input.  Instrumentation only. */
dh2_status dh2_matrix_leaf_split_ms(const dh2_matrix* M, float* ms2);
/* Number of kernels launched by the last dh2_compress (or batched call) that
 * produced M (host int32 out). Instrumentation only: the paper has no
 * counterpart. */
dh2_status dh2_matrix_launch_count(const dh2_matrix* M, int32_t* launches);

/* Kernel classes of dh2_matrix_class_launches (instrumentation only; the paper
 * has no counterpart).  A factor kernel's class is its row class: leaf pairs by
 * cluster size (0: <= 32, 1: <= 40, 2: <= 48, 3: <= 64, 4: more rows),
 * non-leaf pairs by k_t1c' + k_t2c' (0: <= 32, 1: <= 48, 2: <= 64, 3: more). */
enum {
  DH2_KC_LEAF_FACTOR = 0,   /* + leaf row class 0..4: leaf factorisation (Section 6, leaf step)  */
  DH2_KC_LEAF_R = 5,        /* + leaf row class 0..4: R_tc = Q_tc^* G^omega_tc                   */
  DH2_KC_LEVEL_FACTOR = 10, /* + non-leaf row class 0..3: factorisation of Ghat_tc               */
  DH2_KC_LEVEL_R = 14,      /* R_tc = Qhat^* Ghat_tc of a level                                  */
  DH2_KC_NORMS = 15,        /* block norms and nearfield copy                                    */
  DH2_KC_COLW = 16,         /* per-column weights of the leaf column maps                        */
  DH2_KC_CLASSIFY = 17,     /* row classes of a level's non-leaf pairs                           */
  DH2_KC_EXPAND = 18,       /* expansion of non-leaf column bases (Eq. nested)                   */
  DH2_KC_PROJECT = 19,      /* coupling matrices S_b                                             */
  DH2_KC_LEAF_GRAM = 20,    /* + leaf row class 0..3: tensor-core Gram matrices (MIXED_BF16X3)   */
  DH2_KC_GRAM_SCALES = 24,  /* row scales of the leaf Gram matrices (MIXED_BF16X3)               */
  DH2_KC_LEAF_JACOBI = 25,  /* + leaf row class 0..3: Jacobi, rank and Q after the Cholesky (MIXED) */
  DH2_KC_LEAF_R_TC = 29,    /* leaf R_tc = Q_tc^* G^omega_tc on the tensor cores, all classes (MIXED) */
  DH2_KC_COUNT = 32
};
/* Launches of the last compression that produced M, by kernel class
 * (counts: host, DH2_KC_COUNT int32 entries; unused classes are 0). */
dh2_status dh2_matrix_class_launches(const dh2_matrix* M, int32_t* counts);

/* Test instrumentation (the paper has no counterpart): the nth device
 * allocation the library makes from now on (every cudaMalloc and
 * cudaMallocAsync it issues: tree upload, matrix arena, schedule lists,
 * host-input staging buffer, matrix-vector scratch) is refused as if the
 * device were out of memory, so that the failure path of each entry point can
 * be checked without exhausting a GPU; the call that meets it returns
 * DH2_ENOMEM with its output handle NULL.  nth = 0 disarms; DH2_EINVAL for
 * nth < 0.  Process-wide, not thread-specific. */
dh2_status dh2_debug_fail_alloc(int32_t nth);

const char* dh2_status_string(dh2_status s);
/* Library version string. */
const char* dh2_version(void);

#ifdef __cplusplus
}
#endif

#endif /* DH2_H */
