/*
 * tblr.h - C ABI of the GB300 (sm_103a) library for tagged compression of
 * strongly admissible uniform Block Low-Rank matrices.
 *
 * Method: "Randomized Block Low-Rank Matrix Compression by Tagging"
 * (arXiv 2501.05528).  The library computes reconstruct_tag (Table 1):
 *   A ~ U Atilde V^T + B,  U = diag(U_i), V = diag(V_j)  (§2.5 eq. uniformBLRfull)
 * where A is a kernel matrix evaluated tile by tile on the GPU (§7.1) or an
 * explicit matrix, U_i and V_j come from tagged sketches (Algorithm 2),
 * Atilde = U^T (A V) (Table 1 step 2) and the near-field blocks B_ij come from
 * 3^d identity probes (§6.1 eq. sparse_struct_ids; Table 1 step 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All pointers are DEVICE pointers unless a parameter says "host".  The
 *   caller owns every buffer; the library never keeps a pointer after a call
 *   returns (tblr_compress_host excepted, see there).  Work is enqueued on the
 *   CUDA stream `stream` (a cudaStream_t passed as void*; NULL = legacy default
 *   stream) and is complete when that stream is synchronised.
 * - Arrays are dense and row-major unless stated otherwise.  "Box-major" order
 *   is the order of points after the stable sort by box (see tblr_tessellate):
 *   box i owns box-major positions offsets[i] .. offsets[i+1]-1 (the paper's I_i).
 * - Every call returns TBLR_OK (0) or a negative status.  Argument errors are
 *   detected on the host before anything is enqueued; CUDA errors are reported
 *   as TBLR_ECUDA.  tblr_last_error() gives a message for the calling thread.
 * - Floating point: FP64 unless the problem selects TBLR_MIXED.  Then the
 *   sketch contraction (tblr_sketch, tblr_apply, tblr_tagged_sketch) and the
 *   coupling's A_ij V_j run on the tensor cores as three-part BF16 products
 *   with FP32 accumulation, U_i^T W and the near field run on the FP32 pipes
 *   with compensated sums, and tag decode, combine and col stay FP64.
 *
 * Symbols used below: d dimension (1..3); n points; b boxes (product of grid);
 * ell = 3^d + 1 + e tag columns; r = k + p; C = ell * r sketch columns per side;
 * S3 = 3^d (neighbour-list stride); m_i = points in box i.
 */
#ifndef TBLR_H
#define TBLR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------------- status */
#define TBLR_OK            0
#define TBLR_EINVAL       -1  /* bad argument (null pointer, size, alignment, range) */
#define TBLR_ECUDA        -2  /* a CUDA runtime call or launch failed */
#define TBLR_EUNSUPPORTED -3  /* valid but not implemented (e.g. a size beyond a kernel's limit) */
#define TBLR_EWORKSPACE   -4  /* caller workspace or output capacity too small */
#define TBLR_ETIMEOUT     -5  /* a device-side wait gave up (see tblr_device_timeouts) */

/* Operator kinds (§7.1 and explicit matrices). */
#define TBLR_KERNEL_LAPLACE2D 1  /* A_pq = log|x_p - x_q|, A_pp = 0 (§7.1)      */
#define TBLR_KERNEL_LAPLACE3D 2  /* A_pq = 1/(4 pi |x_p - x_q|), A_pp = 0       */
#define TBLR_KERNEL_DENSE     3  /* A given explicitly, n x n, original order   */

/* Precision mode (see "Floating point" above). */
#define TBLR_FP64  0
#define TBLR_MIXED 1  /* three-part BF16 tensor-core sketch and coupling; FP32 near field */

/* Near-field reading (§6.1): the paper's identity probe, or the exact block. */
#define TBLR_NEARFIELD_PROBE 0  /* B_ij = sum_{c: colour(c)=colour(j)} (A_ic - U_i At_ic V_c^T)(:, 0:m_j) */
#define TBLR_NEARFIELD_EXACT 1  /* B_ij = A_ij - U_i At_ij V_j^T  (eq. discrepancymatrix) */

/* How tblr_compress forms the samples S_i = sum_j z_ij Y_j(I_i, :).
 * BLACKBOX: the paper's order - sketch Y = A Omega, Z = A^T Psi with the
 *   explicit extended test matrices, then decode and combine (Algorithm 2).
 * TAGGED: decode first, then S = A' G, R = A'^T H with A'(p, q) =
 *   tau_i(c) A(p, q) for p in I_i, q in I_c (tau_i = T z_i).  Equal to the
 *   black-box S and R in exact arithmetic (eq. extend_test_mat: Y_j(I_i) =
 *   sum_c t_cj A_ic G_c), with ell times fewer multiply-adds and near-field
 *   terms weighted by tau_i(c) ~ 0 instead of cancelling between sketches. */
#define TBLR_SKETCH_BLACKBOX 0
#define TBLR_SKETCH_TAGGED   1
/* Flag, or-ed into TBLR_SKETCH_TAGGED: the caller guarantees A = A^T and
 * passes H = G (Psi = Omega).  Then R = S and V = U (the adjoint sketch of
 * the paper coincides with the direct one when A is self-adjoint), so only S
 * is formed, col runs once and V is a copy of U, and the coupling is formed
 * for i <= j with Atilde_ji = Atilde_ij^T (Atilde_ij = U_i^T A_ij U_j).  The
 * near field is unchanged.  Needs the tag-factored sketch. */
#define TBLR_SKETCH_SELFADJOINT 2

/* Choice of the null vector z_i of T(N_i, :) (tblr_decode).
 * PROJECT: the normalised projection of 1/sqrt(ell) onto the null space.
 * MINRATIO: §5.3 - the null vector minimising the aspect ratio of eq.
 *   aspect_ratio inside the PROJECT vector's sign cell on F_i (a per-box
 *   linear program; boxes with a one-dimensional null space keep PROJECT). */
#define TBLR_Z_PROJECT  0
#define TBLR_Z_MINRATIO 1

/* Problem statement: geometry and tessellation, admissibility, rank
 * (Algorithm 2 "Require": a b x b tessellation of a d-dimensional geometry,
 * target rank k; §2.4 oversampling p; §5.3 extra tag columns e). */
typedef struct {
    int32_t d;          /* 1, 2 or 3 */
    int32_t kernel;     /* TBLR_KERNEL_* */
    int64_t n;          /* number of points, 1 .. 2^31-1 */
    int32_t grid[3];    /* boxes per axis; axes >= d must be 1 */
    double  lo[3];      /* bounding box of the regular grid of boxes */
    double  hi[3];      /* (hi > lo on axes < d) */
    int32_t k;          /* target block rank, >= 1 */
    int32_t p;          /* oversampling, >= 0 (the paper uses 10) */
    int32_t e;          /* extra tag columns, >= 0 (the paper uses 3) */
    int32_t precision;  /* TBLR_FP64 or TBLR_MIXED */
    int32_t nearfield;  /* TBLR_NEARFIELD_PROBE or TBLR_NEARFIELD_EXACT */
    int32_t sketch;     /* TBLR_SKETCH_BLACKBOX or TBLR_SKETCH_TAGGED, optionally | TBLR_SKETCH_SELFADJOINT */
    int32_t zrule;      /* TBLR_Z_PROJECT or TBLR_Z_MINRATIO */
} tblr_problem;

/* Sizes that follow from a problem (no device work). */
typedef struct {
    int64_t b;          /* boxes */
    int32_t ell;        /* 3^d + 1 + e */
    int32_t r;          /* k + p */
    int32_t s3;         /* 3^d */
    int32_t reserved;
    int64_t sketch_cols;/* 2 * ell * r: columns of [Omega | Psi] and of [Y | Z] */
} tblr_sizes;

/* Tessellation arrays (all device, filled by tblr_tessellate). */
typedef struct {
    int32_t *perm;      /* [n]   original index of the point at each box-major position */
    int32_t *box_of;    /* [n]   box of the point at each box-major position */
    int32_t *offsets;   /* [b+1] I_i = box-major positions offsets[i] .. offsets[i+1]-1 */
    int32_t *nbr;       /* [b*S3] N_i ascending, box i included; unused slots = -1 */
    int32_t *nnbr;      /* [b]   |N_i| */
    int32_t *colour;    /* [b]   sum_a (q_a mod 3) 3^a: distinct within every N_i */
    double  *pts;       /* [d*n] box-major coordinates, axis-major (x then y then z) */
} tblr_layout;

/* Status text, and the message of the last failing call on this thread. */
const char *tblr_status_string(int status);
const char *tblr_last_error(void);

/* Derived sizes of a problem; TBLR_EINVAL if the problem is malformed. */
int tblr_sizes_of(const tblr_problem *prob, tblr_sizes *out /* host */);

/* ------------------------------------------------ a1: tessellation (§2.5)
 * Box of point x: q_a = clamp(floor((x_a - lo_a)/(hi_a - lo_a) * grid_a), 0,
 * grid_a - 1), box = q_0 + grid_0 (q_1 + grid_1 q_2).  Points are stably
 * sorted by box (input order kept inside a box).  N_i = boxes whose grid
 * coordinates differ from box i's by at most one on every axis (the boxes
 * sharing a boundary with box i, and i itself; §2.5 strong admissibility).
 * points: [n*d] row-major, original order.  ws: device workspace of at least
 * tblr_tessellate_workspace(prob) bytes, 256-byte aligned.  All layout
 * pointers must be non-null.  Limits: b <= 16384.  Integer results are exact. */
size_t tblr_tessellate_workspace(const tblr_problem *prob);
int tblr_tessellate(const tblr_problem *prob, const double *points,
                    const tblr_layout *out, void *ws, size_t ws_bytes, void *stream);

/* Allocation-free tessellation.  The paper has no counterpart: this entry
 * exists for callers that cannot allocate device memory, such as a request
 * loop running under a device-memory budget fixed up front, or code whose
 * device allocator belongs to a host framework it may not call into.  It
 * computes exactly what tblr_tessellate computes, from the same inputs into
 * the same caller-owned outputs, but takes its scratch from one fixed static
 * device array of TBLR_NOALLOC_SCRATCH_BYTES (8 MiB) that every GPU loading
 * the library holds until the process exits.  It never calls cudaMalloc,
 * cudaFree or any allocating routine.
 * - Limit: tblr_tessellate_workspace(prob) must not exceed 8 MiB (roughly
 *   n * 4 + b * ceil(n / 2048) * 4 bytes); larger problems get TBLR_EINVAL
 *   with a message naming the sizes.
 * - The first call on a device looks up the array's device address with that
 *   device current; make that first call before any stream capture.
 * - All calls on a device share the one array, which keeps the last call's
 *   contents: calls that can overlap on the GPU (different streams without
 *   ordering between them) race and give undefined results.  Calls ordered on
 *   one stream are safe. */
#define TBLR_NOALLOC_SCRATCH_BYTES (8 << 20)
int tblr_tessellate_noalloc(const tblr_problem *prob, const double *points,
                            const tblr_layout *out, void *stream);

/* Near-field block offsets: nf_off[i*S3 + s] = start (in doubles) of block
 * B_{i, nbr[i*S3+s]} (m_i x m_j, row-major) in the near-field array, for
 * s < nnbr[i]; unused slots repeat the next start; nf_off[b*S3] = total.
 * nf_off: [b*S3 + 1] int64.  Also writes max_i m_i to *m_max (device int32). */
int tblr_nearfield_offsets(const tblr_problem *prob, const tblr_layout *lay,
                           int64_t *nf_off, int32_t *m_max, void *stream);

/* ------------------------------- a2: extended test matrices (§4.1, Alg. 2)
 * Omega(I_i, j r + q) = T[i, j] G_i(:, q) and Psi likewise with H_i
 * (eq. extend_test_mat).  T: [b*ell]; G, H: [n*r] in ORIGINAL point order
 * (G_i = rows of G of box i's points, in box-major order).  The output is
 * stored K-major: omega_psi[c*n + p] for column c in [0, 2C) (Omega's columns
 * then Psi's) and box-major position p. */
int tblr_test_matrices(const tblr_problem *prob, const tblr_layout *lay,
                       const double *T, const double *G, const double *H,
                       double *omega_psi, void *stream);

/* --------------------------------- black-box apply (§1: x -> Ax, x -> A^T x)
 * Y = A X (adjoint = 0) or Y = A^T X (adjoint = 1) in box-major order, with A
 * generated on the fly from the layout's points (kernels) or read from `dense`
 * (TBLR_KERNEL_DENSE: [n*n] row-major in ORIGINAL point order; NULL otherwise).
 * X is K-major: xt[c*n + p], c < ncols.  Y: y[p*ldy + c], ldy >= ncols.
 * precision: TBLR_FP64 (ws may be NULL) or TBLR_MIXED (kernels only; needs
 * ws of tblr_apply_workspace bytes).  Limits: ncols <= 8192. */
size_t tblr_apply_workspace(const tblr_problem *prob, int64_t ncols, int precision);
int tblr_apply(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
               const double *xt, int64_t ncols, double *y, int64_t ldy, int adjoint,
               int precision, void *ws, size_t ws_bytes, void *stream);

/* --------------------------------------------- a3: sketch (Algorithm 2)
 * [Y | Z] = [A Omega | A^T Psi]: yz[p*2C + c], c < C for Y and C + c for Z,
 * from omega_psi as written by tblr_test_matrices.  Symmetric kernels run both
 * halves in one pass over A.  Uses prob->precision. */
size_t tblr_sketch_workspace(const tblr_problem *prob);
int tblr_sketch(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                const double *omega_psi, double *yz, void *ws, size_t ws_bytes, void *stream);

/* Tag-factored samples (see TBLR_SKETCH_TAGGED): S(I_i, :) = sum_c tau[i, c]
 * A_ic G_c and R(I_i, :) = sum_c tau[i, c] (A^T)_ic H_c directly from the
 * projected tags tau (b x b, from tblr_decode) and G, H ([n*r], original point
 * order).  s, rr: [n*r] box-major.  FP64, or with TBLR_MIXED on the tensor
 * cores (three-part BF16, FP32 accumulation, FP32 tags).  The sketch Y, Z is
 * never formed.  With TBLR_SKETCH_SELFADJOINT only s is written (H and rr may
 * be NULL; R = S).  ws: tblr_tagged_sketch_workspace bytes. */
size_t tblr_tagged_sketch_workspace(const tblr_problem *prob);
int tblr_tagged_sketch(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                       const double *tau, const double *G, const double *H, double *s,
                       double *rr, void *ws, size_t ws_bytes, void *stream);

/* Tile-width autotuner of the mixed-precision tag-factored sketch (TBLR_MIXED
 * with a built-in kernel).  Runs tblr_tagged_sketch with each admissible
 * tensor-core tile width (32, 64, 96, 128, 160 columns, at most 64 padded
 * columns beyond the 32-column round-up of the sketch columns), timing two
 * runs after a warm-up with CUDA events on `stream` (so it synchronises the
 * stream and must not be captured in a graph), and records the fastest width
 * for this process under (kernel, sketch columns, floor(log2 n)); later
 * tagged sketches of that class use it, including ones captured into graphs.
 * Arguments as tblr_tagged_sketch; *width (host) receives the chosen width and
 * s (and rr) hold that width's result.  tblr_tuned_width gives the width the
 * class currently uses (0: the built-in rule: fewest tiles of at most 160
 * columns); tblr_tune_clear forgets every recorded width. */
int tblr_tune_tagged_sketch(const tblr_problem *prob, const tblr_layout *lay, const double *tau,
                            const double *G, const double *H, double *s, double *rr, void *ws,
                            size_t ws_bytes, int32_t *width /* host */, void *stream);
int tblr_tuned_width(const tblr_problem *prob, int32_t *width /* host */);
void tblr_tune_clear(void);

/* ------------------------------------ a4: tag decode (§4.1, §5.1, §5.3)
 * z_i = unit vector of null(T(N_i, :)) nearest to 1/sqrt(ell) (the normalised
 * projection of the all-ones direction; eq. tagsubmat), tau_i = T z_i (projected
 * tags), rho_i = max |tau_i(F_i)| / min |tau_i(F_i)| (eq. aspect_ratio; NaN when
 * F_i is empty).  z: [b*ell], tau: [b*b] (tau[i*b + q]), rho: [b].
 * With prob->zrule = TBLR_Z_MINRATIO each box then solves the §5.3 linear
 * program (see TBLR_Z_MINRATIO) on the GPU in FP64; a box whose program stops
 * without an optimum (an iteration cap) keeps the projected vector and is
 * counted by tblr_decode_lp_failures.  Limits: ell <= 32. */
int tblr_decode(const tblr_problem *prob, const tblr_layout *lay, const double *T,
                double *z, double *tau, double *rho, void *stream);
/* Boxes whose §5.3 program stopped without an optimum since the last call
 * (synchronises the device, then resets the count). */
int tblr_decode_lp_failures(unsigned int *count /* host */);

/* Algorithm 3 (the plain per-box randomized range finder, §4.2 "basic") on the
 * same machinery: tau[i*b + c] = 0 for c in N_i and 1 otherwise (b x b FP64).
 * tblr_tagged_sketch with this tau gives S(I_i, :) = A(I_i, F_i) G(F_i) and
 * R(I_i, :) = A(F_i, I_i)^T H(F_i), Algorithm 3's samples with one shared
 * Gaussian G (H) restricted to each far field, and tblr_col turns them into
 * its bases.  With kernel operators this costs the tag-factored sketch's
 * N^2 2r multiply-adds; as black-box matvecs Algorithm 3 needs 2 b r. */
int tblr_far_indicator(const tblr_problem *prob, const tblr_layout *lay, double *tau,
                       void *stream);

/* ------------------------------ a5: combine (Algorithm 2; eq. projected_tags)
 * S(I_i, :) = sum_j z_ij Y(I_i, j r : (j+1) r), R likewise from Z.
 * yz: [n*2C]; s, rr: [n*r]. */
int tblr_combine(const tblr_problem *prob, const tblr_layout *lay, const double *yz,
                 const double *z, double *s, double *rr, void *stream);

/* ---------------------------------------------- a6: col (§2.3, §2.4)
 * U(I_i, 0:k_i) = k_i dominant left singular vectors of S(I_i, :), each column
 * signed so its largest-magnitude entry is positive (lowest index on ties);
 * columns k_i..k-1 are zero.  k_i = min(k, m_i), or 0 when F_i is empty.
 * Method: FP64 Householder QR; one-sided Jacobi SVD of R in FP32, its
 * rotations re-orthonormalised in FP64 and polished by FP64 sweeps; Q applied
 * back in FP64.
 * s: [n*r]; u: [n*k]; ranks: [b] (written).  ws: tblr_col_workspace bytes.
 * Limits: r <= 112. */
size_t tblr_col_workspace(const tblr_problem *prob);
int tblr_col(const tblr_problem *prob, const tblr_layout *lay, const double *s,
             double *u, int32_t *ranks, void *ws, size_t ws_bytes, void *stream);

/* ---------------------------------- a7: coupling (Table 1 step 2, §2.5)
 * Atilde_ij = U_i^T A_ij V_j for ALL box pairs: at[((i*b + j)*k + a)*k + c],
 * zero outside a < k_i, c < k_j.  u, v: [n*k]; ranks: [b]; m_max = max_i m_i
 * (as returned by tblr_nearfield_offsets).  FP64, or with TBLR_MIXED on the
 * tensor cores: A_ij V_j as three-part BF16 products with FP32 accumulation
 * per 64-point chunk and compensated sums, then U_i^T W in FP32 with
 * compensated sums (~1e-7 relative; the environment variable
 * TBLR_COUPLING_SIMT=1 selects an FP32 SIMT form of the same sums).  With
 * TBLR_SKETCH_SELFADJOINT the caller passes v = u (A = A^T) and only i <= j
 * are formed, Atilde_ji = Atilde_ij^T.
 * ws: tblr_coupling_workspace bytes (0 for FP64; with TBLR_MIXED the points
 * and U in a per-box padded order, the BF16 parts of V and a status word),
 * 256-byte aligned.  A device-side wait that times out makes the output
 * undefined and is counted by tblr_device_timeouts.
 * Limits: k <= 64; mixed: b <= 65535 and n < 2^30 (the SIMT form also
 * m_max <= ~780). */
size_t tblr_coupling_workspace(const tblr_problem *prob);
int tblr_coupling(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                  const double *u, const double *v, const int32_t *ranks, int32_t m_max,
                  double *at, void *ws, size_t ws_bytes, void *stream);

/* ------------------ a8: near field (Table 1 step 3; §6.1 eq. sparse_struct_ids)
 * For every neighbour pair (i, j = nbr[i*S3+s]) writes B_ij (m_i x m_j,
 * row-major) at bnear + nf_off[i*S3+s], using prob->nearfield's reading.
 * ws: tblr_nearfield_workspace(prob, m_max) bytes. */
size_t tblr_nearfield_workspace(const tblr_problem *prob, int32_t m_max);
int tblr_nearfield(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                   const double *u, const double *at, const double *v, const int32_t *ranks,
                   const int64_t *nf_off, int32_t m_max, double *bnear,
                   void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------------- whole pipeline (Table 1)
 * Runs a2..a8 on a tessellated problem (tblr_tessellate and
 * tblr_nearfield_offsets already enqueued; m_max is their host-read value).
 * Outputs as in the step calls: yz [n*2C] (kept for inspection; unused and
 * may be NULL with TBLR_SKETCH_TAGGED), z, tau, rho,
 * u, v [n*k], ranks [b], at [b*b*k*k], bnear [nf_off[b*S3]].  Scratch (Omega,
 * S, R and the steps' workspaces) comes from ws, tblr_compress_workspace bytes. */
size_t tblr_compress_workspace(const tblr_problem *prob, int32_t m_max);
int tblr_compress(const tblr_problem *prob, const tblr_layout *lay, const double *dense,
                  const double *T, const double *G, const double *H,
                  double *yz, double *z, double *tau, double *rho,
                  double *u, double *v, int32_t *ranks, double *at,
                  const int64_t *nf_off, int32_t m_max, double *bnear,
                  void *ws, size_t ws_bytes, void *stream);

/* ------------------------------------- end to end from HOST buffers
 * The same compression with every input and output in host memory: copies
 * points, T, G, H (and dense) to the device, tessellates, runs the pipeline
 * and copies perm, offsets, nbr, ranks, U, V, Atilde and B back, all on
 * `stream`, and synchronises it before returning.  Device memory is taken
 * from a per-device cache owned by the library (grown on demand, freed by
 * tblr_release_device_cache).  Host output sizes: perm [n], offsets [b+1],
 * nbr [b*S3], ranks [b], u, v [n*k], at [b*b*k*k] (doubles/ints); bnear has
 * room for bnear_capacity doubles.  *bnear_size receives the doubles B needs;
 * if that exceeds bnear_capacity, nothing else is copied and the call returns
 * TBLR_EWORKSPACE.  Pinned host buffers make the copies asynchronous. */
int tblr_compress_host(const tblr_problem *prob, const double *points_h,
                       const double *T_h, const double *G_h, const double *H_h,
                       const double *dense_h,
                       int32_t *perm_h, int32_t *offsets_h, int32_t *nbr_h,
                       int32_t *ranks_h, double *u_h, double *v_h, double *at_h,
                       double *bnear_h, int64_t bnear_capacity, int64_t *bnear_size,
                       void *stream);
int tblr_release_device_cache(void);

/* Device-side waits of the tensor-core kernels (mbarrier pipelines) are
 * bounded: a wait that does not complete within ~0.5 s abandons its launch,
 * whose output is then undefined, and increments a per-device counter.  This
 * call synchronises the device, stores the counter in *count, resets it, and
 * returns TBLR_OK (or TBLR_ECUDA). */
int tblr_device_timeouts(unsigned int *count /* host */);

/* ------------------------------------------------------- batched jobs
 * Independent compressions with uneven sizes, box sizes, ranks and
 * dimensions run together: every job's pipeline is enqueued on one of
 * n_streams worker streams (largest estimated sketch work first, to the least
 * loaded stream), forked from and joined back into `stream` with events, with
 * no host synchronisation, so the batch can be captured into one CUDA graph.
 * A job's buffers are caller-owned device memory sized as for the step calls;
 * ws must hold max(tblr_tessellate_workspace, tblr_compress_workspace(m_max)).
 * tblr_batch_plan tessellates each job once (synchronising `stream`) and fills
 * m_max and nf_total; tblr_batch_run then requires the same points (the
 * near-field sizes depend on them). */
typedef struct {
    tblr_problem prob;
    const double *points, *T, *G, *H, *dense;   /* inputs (dense: TBLR_KERNEL_DENSE only) */
    tblr_layout lay;                             /* tessellation outputs */
    int64_t *nf_off;                             /* [b*S3 + 1] */
    int32_t *m_max_dev;                          /* [1] */
    int32_t m_max;                               /* filled by tblr_batch_plan */
    int32_t reserved;
    int64_t nf_total;                            /* filled by tblr_batch_plan */
    double *yz, *z, *tau, *rho, *u, *v;          /* outputs as in tblr_compress */
    int32_t *ranks;
    double *at, *bnear;
    void *ws;
    size_t ws_bytes;
} tblr_job;

int tblr_batch_plan(int n_jobs, tblr_job *jobs, void *stream);
int tblr_batch_run(int n_jobs, const tblr_job *jobs, int n_streams, void *stream);

/* A captured batch: tblr_graph_create records tblr_batch_run on `stream`
 * (which must not be the legacy default stream) into a CUDA graph;
 * tblr_graph_launch replays the whole batch with one launch. */
typedef struct tblr_graph tblr_graph;
int tblr_graph_create(int n_jobs, const tblr_job *jobs, int n_streams, void *stream,
                      tblr_graph **out);
int tblr_graph_launch(tblr_graph *graph, void *stream);
void tblr_graph_destroy(tblr_graph *graph);

/* ------------------------------------------------------------ serving
 * A continuous-batching server.  Requests queue in arrival order; a request
 * is admitted when one of max_inflight stream slots is free and its
 * first-phase device memory (inputs, tessellation) fits in mem_budget_bytes;
 * its second phase (the pipeline and outputs), sized exactly after
 * tessellation, starts when that memory fits too (a request that alone
 * exceeds the budget runs when nothing else compresses).  Admitted requests
 * run on their own streams and overlap on the device; results do not depend
 * on what runs beside them.  Inputs and outputs are host buffers owned by the
 * caller and must stay valid until tblr_server_wait returns (pinned memory
 * makes the copies asynchronous).  Output sizes are those of
 * tblr_compress_host; a request whose near field exceeds bnear_capacity
 * finishes with status TBLR_EWORKSPACE.  Kernel operators only. */
typedef struct {
    tblr_problem prob;
    const double *points_h, *T_h, *G_h, *H_h;
    int32_t *perm_h, *offsets_h, *nbr_h, *ranks_h;
    double *u_h, *v_h, *at_h, *bnear_h;
    int64_t bnear_capacity;
} tblr_request;

typedef struct {
    uint64_t completed, failed, pending, active;
    double p50_ms, p99_ms;      /* submit-to-done latency of completed requests */
    double throughput;          /* completed / (last completion - first submit), per second */
    size_t mem_in_use, mem_peak;
} tblr_server_report;

typedef struct tblr_server tblr_server;
int tblr_server_create(tblr_server **out, int device, size_t mem_budget_bytes, int max_inflight);
int tblr_server_submit(tblr_server *server, const tblr_request *req, uint64_t *ticket);
/* Waits up to timeout_ms for a request; TBLR_ETIMEOUT if it is not done yet
 * (the request keeps running; wait again).  *status is the request's own
 * result status.  The ticket is released when this returns TBLR_OK. */
int tblr_server_wait(tblr_server *server, uint64_t ticket, int timeout_ms, int *status,
                     double *latency_ms);
int tblr_server_stats(tblr_server *server, tblr_server_report *out);
/* Finishes every queued and running request, then frees the server. */
void tblr_server_destroy(tblr_server *server);

#ifdef __cplusplus
}
#endif
#endif /* TBLR_H */
