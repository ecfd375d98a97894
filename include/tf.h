/*
 * tf.h -- C ABI of the GB300 BTTB/BCCB sensitivity-product library (libtf.so).
 *
 * The library applies the sensitivity matrix G of potential-field inversion and its
 * transpose to vectors and blocks of vectors (Renaut, Hogue & Vatankhah, "Fast
 * focusing inversion of gravity and magnetic data...", arXiv:2004.13904):
 *
 *   G = [G^(1), ..., G^(nz)]                           (Sec. 2.1, Eq. (3))
 *   each G^(r) is BTTB; it is embedded in a BCCB matrix whose first column, reshaped to
 *   T_r of size (sx+nx-1) x (sy+ny-1), has the precomputed 2-D FFT  G^_r  (App. A);
 *   G x   = sum_r extract(ifft2(G^_r .* fft2(pad(x^(r)))))   (App. A)
 *   G^T y = [extract(ifft2(conj(G^_r) .* fft2(pad(y))))]_r    (App. A, last paragraph)
 *   G~ x  = W_d (G (W^-1 x))                                  (Sec. 2.5, Eq. (10))
 *
 * Geometry (Sec. 2.1, Fig. 1): cells are indexed 0<=p<nx, 0<=q<ny, 0<=r<nz with
 * nx = sx+pxl+pxr, ny = sy+pyl+pyr; cell p spans [p dx, (p+1) dx]; station (i,j) sits at
 * height station_z over the centre of cell (i+pxl, j+pyl); layer r spans
 * [z_edges[r], z_edges[r+1]] with z positive down.  m = sx*sy, n = nx*ny*nz.
 * Vectors: model x has index p + nx*(q + ny*r); data d has index i + sx*j.
 * Blocks are column-major: column b of X starts at X + b*ldx.
 *
 * Conventions for every call:
 *  - every function returns a tf_status; tf_last_error() gives a message for the
 *    last failure on the calling thread (library-owned string).  Nothing throws.
 *  - vectors and blocks are DEVICE pointers owned by the caller, of the operator's
 *    dtype (float for TF_F32, double for TF_F64), on the device that was current when
 *    the operator was created; that device must be current for every call.
 *  - products are asynchronous and ordered on the caller's stream (a cudaStream_t
 *    passed as tf_stream; NULL = legacy default stream).  Inputs must not alias outputs.
 *  - the operator owns its spectra and a workspace; calls on one operator must be
 *    ordered (one stream, or caller-side synchronisation).  Different operators are
 *    independent.
 *  - colscale (length n) and rowscale (length m) are optional diagonal scalings;
 *    NULL means identity.
 */
#ifndef TF_H
#define TF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TF_OK = 0,
  TF_EINVAL = 1,        /* invalid argument (null pointer, bad size, bad geometry)   */
  TF_ENOMEM = 2,        /* device allocation failed                                  */
  TF_ECUDA = 3,         /* a CUDA runtime call or kernel launch failed               */
  TF_EUNSUPPORTED = 4,  /* valid but outside what the library supports (FFT size)   */
  TF_ENOTCONV = 5,      /* reserved for iterative drivers                            */
  TF_ETIMEOUT = 6       /* a bounded device-side wait ran out (tf_batch_persistent;  */
                        /* the product kernels' copy waits, reported by tf_destroy)  */
} tf_status;

typedef enum { TF_F32 = 0, TF_F64 = 1 } tf_dtype;

typedef void* tf_stream; /* a cudaStream_t */

/* Station/volume geometry (Sec. 2.1, Fig. 1; padding counts per side, Sec. 3.2). */
typedef struct {
  int sx, sy;                 /* stations along x and y (>= 1)                         */
  int nz;                     /* depth layers (>= 1)                                    */
  int pxl, pxr, pyl, pyr;     /* padding cells per side (>= 0), no stations over them   */
  double dx, dy;              /* cell sizes in metres (> 0)                             */
  const double* z_edges;      /* HOST array of nz+1 strictly increasing depths (m)      */
  double station_z;          /* station depth (m), <= z_edges[0]                        */
} tf_grid;

typedef struct tf_op tf_op;

/* Build the layer spectra G^_r of the vertical-attraction kernel (Sec. 2.1, Eq. (3);
 * App. A "the 2DFFT of T is precomputed").  Units: mGal per g/cc.  The kernel table and
 * its 2-D FFT are evaluated on the device in FP64; for TF_F32 the spectra are then
 * rounded once to FP32.  Blocks the calling thread until the set-up is complete.
 * Errors: TF_EINVAL (null pointers, sizes < 1, negative padding, non-increasing
 * z_edges, station below the top of the volume), TF_EUNSUPPORTED (embedding larger
 * than 1024 along x or y), TF_ENOMEM, TF_ECUDA.  On error *out is set to NULL. */
tf_status tf_create_gravity(const tf_grid* grid, tf_dtype dtype, tf_stream stream, tf_op** out);

/* Same for the total-field anomaly of induced magnetisation without remanence or
 * self-demagnetisation (Sec. 2.1): inclination/declination in degrees of the inducing
 * field (x north, y east, z down) and its strength in nT.  Units: nT per SI. */
tf_status tf_create_magnetic(const tf_grid* grid, double inc_deg, double dec_deg,
                             double field_nt, tf_dtype dtype, tf_stream stream, tf_op** out);

/* Release the operator and everything it owns (waits for the device's work to finish).
 * NULL is accepted.  Returns TF_ECUDA if that wait reports a fault of earlier work, and
 * TF_ETIMEOUT if a product kernel's bounded wait for one of its asynchronous copies ran
 * out (about 2 s; that kernel's outputs are then incomplete; the record is cleared); the
 * operator is released either way. */
tf_status tf_destroy(tf_op* op);

/* m = sx*sy, n = nx*ny*nz. */
tf_status tf_dims(const tf_op* op, int64_t* m, int64_t* n);

/* FFT sizes chosen for the embedding: n1 >= sx+nx-1, n2 >= sy+ny-1 (any such size gives
 * the exact product, because T is zero beyond the minimum size). */
tf_status tf_fft_dims(const tf_op* op, int* n1, int* n2);

/* d = diag(rowscale) G diag(colscale) x   (Sec. 2.5 Eq. (10); App. A)
 * x: n values, d: m values.  Errors: TF_EINVAL (null x/d or op), TF_ECUDA. */
tf_status tf_matvec(tf_op* op, const void* x, void* d, const void* colscale,
                    const void* rowscale, tf_stream stream);

/* x = diag(colscale) G^T diag(rowscale) y   (App. A, last paragraph)
 * y: m values, x: n values. */
tf_status tf_rmatvec(tf_op* op, const void* y, void* x, const void* colscale,
                     const void* rowscale, tf_stream stream);

/* D = diag(rowscale) G diag(colscale) X for B columns (Sec. 2.5: block products are
 * loops over columns; here the spectra are shared by the whole block).
 * X: column b at X + b*ldx (ldx >= n); D: column b at D + b*ldd (ldd >= m).
 * B = 0 is a no-op.  Errors: TF_EINVAL (B < 0, ldx < n, ldd < m, null pointers). */
tf_status tf_matmat(tf_op* op, int64_t B, const void* X, int64_t ldx, void* D, int64_t ldd,
                    const void* colscale, const void* rowscale, tf_stream stream);

/* X = diag(colscale) G^T diag(rowscale) Y for B columns; Y: ldy >= m, X: ldx >= n.
 * (X^T G^T = (G X)^T and Y^T G = (G^T Y)^T need no further entry, App. A.) */
tf_status tf_rmatmat(tf_op* op, int64_t B, const void* Y, int64_t ldy, void* X, int64_t ldx,
                     const void* colscale, const void* rowscale, tf_stream stream);

/* D = diag(rowscale) G diag(colscale) X for B1 columns and XT = diag(colscale) G^T
 * diag(rowscale) Y for B2 columns, from and to HOST memory, with the copies inside the
 * call (App. A, as tf_matmat / tf_rmatmat).  X (ldx >= n), D (ldd >= m), Y (ldy >= m) and
 * XT (ldxt >= n) are host pointers to column-major blocks; either product may be empty
 * (B = 0, its pointers may then be NULL); colscale / rowscale are DEVICE vectors or NULL.
 * The columns go through the device in `chunks` chunks (>= 1): the host-to-device copy of
 * one chunk, the products of another and the device-to-host copy of a third overlap on two
 * internal copy streams and the caller's stream, with G^T's chunks ahead of G's so that
 * the two large copies (X in, XT out) use both directions of the host link at once.
 * Device staging (three slots per product, each one chunk's input and output) is kept in
 * the operator and grown on demand (growth frees and allocates device memory).  The call
 * is stream-ordered: the copies start after the work already queued on `stream`, and
 * `stream` continues after the last copy out, so the caller synchronises `stream` before
 * reading D or XT.  Copies overlap only from page-locked host memory.  The host blocks
 * must not change before that point.  Errors: TF_EINVAL (negative B, chunks < 1, NULL
 * block of a non-empty product, leading dimension below the rows), TF_ENOMEM, TF_ECUDA. */
tf_status tf_products_host(tf_op* op, int64_t B1, const void* X, int64_t ldx, void* D,
                           int64_t ldd, int64_t B2, const void* Y, int64_t ldy, void* XT,
                           int64_t ldxt, const void* colscale, const void* rowscale, int chunks,
                           tf_stream stream);

/* Copy the operator's layer spectra, nz x n2 x (n1/2+1) complex values of its dtype
 * (interleaved re/im, k1 fastest), already divided by n1*n2, to dst (device or host
 * memory; bytes must equal that size).  Ordered on stream.  For checks and tools. */
tf_status tf_get_spectra(const tf_op* op, void* dst, int64_t bytes, tf_stream stream);

/* Tuning knobs of the product kernels: rows-stage sequence pairs per CTA (4, 8, 16) and
 * column-stage k1 columns per CTA (4, 8, 16) of the generic engine (the compile-time
 * plans have fixed tiles), and columns per workspace chunk (>= 1; the workspace is
 * reallocated to exactly that many columns and no longer grows).  0 keeps the current
 * value.  By default the workspace grows, on the first product with more columns than
 * it holds, up to the columns that fit in 16 GiB, or in an eighth of the device memory
 * free when the operator was created if that is less (the growth frees and allocates
 * device memory, which waits for the device to be idle); a block is processed in the
 * fewest chunks of equal size.  Must not be called while products of this operator are
 * in flight. */
tf_status tf_set_tuning(tf_op* op, int rows_tile, int cols_tile, int64_t chunk_cols);
tf_status tf_get_tuning(const tf_op* op, int* rows_tile, int* cols_tile, int64_t* chunk_cols);

/* FFT engine of the product kernels: 0 (default) uses compile-time plans for the
 * transform lengths that have one (32, 64, 96, 128, 160, 192, 224, 256, 320, 448, 512)
 * and the generic engine otherwise; 1 forces the generic engine.  Both compute the same
 * product.  tf_get_engine also reports whether the row (x) and column (y) transforms
 * currently run on compiled plans. */
tf_status tf_set_engine(tf_op* op, int engine);
tf_status tf_get_engine(const tf_op* op, int* engine, int* compiled_rows, int* compiled_cols);

/* Per-stage timing with CUDA events recorded around every stage launch on the call's
 * stream.  Enable (1) / disable (0) clears the record.  tf_profile_read synchronises
 * on the recorded events and returns, for the stages
 *   0 rows_r2c (model rows), 1 cols_fwd, 2 rows_c2r (data rows),
 *   3 rows_r2c (data rows),  4 cols_adj, 5 rows_c2r (model rows),
 * the total milliseconds, the number of launches and the columns processed
 * (arrays of length 6). */
tf_status tf_profile_enable(tf_op* op, int enable);
tf_status tf_profile_read(tf_op* op, double* ms, int64_t* launches, int64_t* columns);

/* d = diag(rowscale) G diag(colscale) x for one column, as tf_matvec computes it, but
 * without allocating anything.  The paper has no counterpart: this entry point exists for
 * callers that cannot call cudaMalloc when they run the product -- for example code
 * running under a memory budget that forbids new device allocations, or between points
 * where an allocator must not be entered.  The operator itself must have been created
 * beforehand (creation allocates).  Instead of the operator's workspace the call uses a
 * fixed 8 MiB scratch buffer compiled into the library (a __device__ array that a device
 * holds from the creation of the first operator on it until the process exits).
 *  - Operator creation (tf_create_*) looks up the buffer's address on its device and
 *    loads the kernels this call launches, so the call itself loads no code and makes no
 *    allocation, on its first use as on any later one.  The current device must be the
 *    operator's.
 *  - The call always runs the generic FFT engine (whatever tf_set_engine selected), so
 *    its result agrees with tf_matvec's within the product tolerances, not bitwise.
 *  - All calls share the one buffer, which keeps the previous call's contents; the
 *    kernels read it only at positions written earlier in the same call.  Calls that
 *    overlap on the GPU -- on different streams, or from different host threads without
 *    ordering -- race on the buffer and give wrong results.
 *  - Errors: TF_EINVAL if the operator needs more than 8 MiB of scratch for one column
 *    ((nz*ny + n2)*hs + (sy + n2)*hs complex values of its dtype, hs = n1/2+1 rounded up
 *    to a multiple of 16, plus alignment), if x or d is NULL, or if another device is
 *    current; TF_ECUDA if a launch fails. */
tf_status tf_matvec_noalloc(const tf_op* op, const void* x, void* d, const void* colscale,
                            const void* rowscale, tf_stream stream);

/* Bounds checking (debug builds).  In a library compiled with -DTF_BOUNDS_CHECK
 * (libtf_checked.so), every global access of the product kernels is tested against its
 * buffer's extent and skipped when outside it; the first violation is recorded.  This
 * call returns and clears that record: *checked = 1 in a checked build (else 0), *site
 * identifies the access (0 = none recorded), *offset and *extent its element offset
 * within the column's buffer and that buffer's length.  Synchronises the device. */
tf_status tf_debug_oob(int* checked, int* site, int64_t* offset, int64_t* extent);

/* Gram-Schmidt helpers for the projected solvers (Alg. 1 re-orthogonalisation; the
 * paper uses MGS, these give one classical pass, applied twice for CGS2, or one MGS
 * step with k = 1).  A is a stack of k vectors of length len, vector j at A + j*lda
 * (dtype elements), DEVICE memory.
 * tf_rows_dot:  y[j] = A_j . x for j < k; y is a DEVICE double[k].
 * tf_rows_axpy: x -= sum_j c[j] A_j; c is a DEVICE double[k].
 * Sums are accumulated in FP64 for TF_F64 data and in double-float arithmetic (pairs of
 * floats combined with exact TwoSum/TwoProd steps, about 44 significant bits) for TF_F32
 * data, which keeps them on the FP32 pipe.
 * Deterministic (fixed reduction order), stream-ordered.  Errors: TF_EINVAL. */
tf_status tf_rows_dot(tf_dtype dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                      const void* x, double* y, tf_stream stream);
tf_status tf_rows_axpy(tf_dtype dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                       const double* c, void* x, tf_stream stream);

/* Measured arithmetic peak of the current device for dtype: a launch of 8 CTAs per SM,
 * 256 threads each running 8 independent fused multiply-add chains, timed with CUDA
 * events; *tflops = 2 flop x FMAs / time.  The denominator of ALU-bound rooflines.
 * Synchronises the stream.  Errors: TF_EINVAL, TF_ENOMEM, TF_ECUDA. */
tf_status tf_peak_probe(tf_dtype dtype, double* tflops, tf_stream stream);

/* ---- IRLS focusing inversion drivers (Sec. 2.3, Alg. 1, Alg. 2, Sec. 3.1) -------------
 *
 * Both drivers minimise the focusing functional of Eq. (4) by iteratively reweighted
 * least squares on the operator's products:
 *   W = W_z W_L^(k), W_z = diag(zbar_r^(-beta)) per layer (zbar_r the mean depth of layer
 *   r below the stations), W_L^(1) = I, (W_L^(k))_ii = ((m_i^(k-1) - m_i^(k-2))^2 +
 *   eps2)^((lam - 2)/4);  G~ = W_d G W^-1 with W_d = diag(1/sigma)  (Eq. (10));
 *   r~ = W_d (d_obs - G m^(k-1));  the projected problem gives z with
 *   min ||G~ z - r~||^2 + alpha^2 ||z||^2;  m^(k) = clip(m^(k-1) + W^-1 z, lower, upper);
 *   alpha^(1) from Eq. (11) (mean over the t retained singular values above 1e-14 s_1),
 *   alpha^(k>1) minimises UPRE for whitened noise on the t retained terms (a 200-point
 *   log grid on [max(s_t, 1e-14 s_1)/10, s_1], then 80 golden-section steps in log alpha
 *   between the best point's neighbours);  stop after kmax iterations or, with chi2_stop,
 *   once ||W_d (G m^(k) - d_obs)||^2 <= m + sqrt(2 m)  (Eq. (12)).
 * tf_gkb projects with t_p steps of Golub-Kahan bidiagonalisation of G~ started from r~
 * (Alg. 1) with re-orthogonalisation of both bases (classical Gram-Schmidt applied
 * twice, or modified Gram-Schmidt), UPRE on the t largest singular values of the
 * (t_p+1) x t_p bidiagonal B (from its Golub-Kahan tridiagonal form), and the Tikhonov
 * solution on all t_p terms, i.e. the least squares solution of
 * [B; alpha I] y = [||r~|| e_1; 0] (Givens QR), z = A y.
 * tf_rsvd projects with the randomised SVD of Alg. 2 with one power iteration from the
 * caller's Gaussian test matrix Omega, keeps the t largest singular values of B = G~ Q
 * (eigen-decomposition of B^T B) and z = Q V_t Gamma(alpha) U_t^T r~.
 *
 * Arguments: d_obs, sigma (length m) and m_out (length n) are DEVICE arrays of the
 * operator's dtype; omega (tf_rsvd) is a DEVICE t_p x m array, row-major (row j = the j-th
 * test vector).  m_out receives m^(K), the last iterate (m^(0) = 0).  The drivers
 * allocate their own device workspace (A: t_p x n and H: (t_p+1) x m for tf_gkb; five
 * t_p x max(n, m) blocks for tf_rsvd), run on `stream`, and synchronise it before
 * returning.  The projected problems are solved on the host in FP64.  tf_rsvd uses
 * cuSOLVER (QR, symmetric eigen-decomposition) and cuBLAS (B^T B); a basis block above
 * 2^30 values (c4: 10^6 x 2510) is factored as a tall-skinny QR of row blocks below that
 * size, which needs two more buffers of one row block each.  Errors: TF_EINVAL
 * (bad sizes or parameters, t > t_p, tf_rsvd with t_p > min(m, n)), TF_ENOMEM, TF_ECUDA,
 * TF_ENOTCONV (the host eigenvalue iteration did not converge). */
typedef struct {
  int t;              /* retained terms, 1 <= t <= tp                                 */
  int tp;             /* projected size t_p                                           */
  double beta;        /* depth-weighting exponent (0.8 gravity, 1.4 magnetic, Sec. 3) */
  double lam;         /* focusing norm (1: approximately L1, Sec. 2.2)                */
  double eps2;        /* focusing parameter epsilon^2 (> 0)                           */
  double lower, upper;/* bounds on the model                                          */
  int kmax;           /* maximum number of IRLS iterations (>= 1)                     */
  int chi2_stop;      /* nonzero: stop on Eq. (12)                                    */
  int reorth;         /* tf_gkb: 0 = classical Gram-Schmidt twice, 1 = modified       */
  const double* alphas; /* HOST, kmax entries, or NULL: fixed alpha^(k) (skips UPRE)  */
} tf_irls_params;

typedef struct {
  int iterations;     /* iterations run                                               */
  double* alpha;      /* HOST arrays of kmax entries (each may be NULL): alpha^(k),  */
  double* chi2;       /*   chi^2 of m^(k), and seconds of iteration k                 */
  double* seconds;
} tf_irls_report;

tf_status tf_gkb(tf_op* op, const tf_irls_params* params, const void* d_obs, const void* sigma,
                 void* m_out, tf_irls_report* report, tf_stream stream);
tf_status tf_rsvd(tf_op* op, const tf_irls_params* params, const void* d_obs, const void* sigma,
                  const void* omega, void* m_out, tf_irls_report* report, tf_stream stream);

/* ---- batches of independent problems (uneven sizes) ------------------------------------
 *
 * A tf_batch groups `count` operators (any mix of grids, kinds and dtypes on the current
 * device) whose block products are independent.  tf_batch_products computes, for every
 * i < count with non-NULL pointers, D[i] = G_i X[i] and XT[i] = G_i^T Y[i] on B columns
 * (X[i]: n_i x B with ld n_i, D[i]: m_i x B with ld m_i, Y[i]: m_i x B, XT[i]: n_i x B;
 * DEVICE pointers of operator i's dtype), spreading the operators over `streams`
 * internal streams forked from and joined back into `stream`, so that problems too small
 * to fill the GPU run side by side.  With use_graph, the first call with a given
 * (B, pointer arrays, operator workspaces) runs eagerly, the next records the forked
 * launches as one CUDA graph, and later identical calls replay it (one launch); any
 * change re-records.  Operators must not be used elsewhere while a batch call runs.
 * The batch does not own the operators.  Errors: TF_EINVAL, TF_ENOMEM, TF_ECUDA, and
 * the products' errors.  (Batched products of many problems, App. A applied per problem.) */
typedef struct tf_batch tf_batch;
tf_status tf_batch_create(tf_op* const* ops, int count, int streams, tf_batch** out);
tf_status tf_batch_destroy(tf_batch* batch);
tf_status tf_batch_products(tf_batch* batch, int64_t B, const void* const* X, void* const* D,
                            const void* const* Y, void* const* XT, int use_graph, tf_stream stream);

/* One persistent launch for the whole batch (App. A applied per problem).  Every
 * operator's G X and G^T Y (as in tf_batch_products; operators of one dtype) run in a
 * single kernel over a work list of column tiles: resident CTAs claim tiles in order from
 * a device counter, rows stage before column stage before rows stage for each problem,
 * direction and column, on the generic FFT engine (each operator's radix plans, see
 * tf_set_radices).  The batch owns a workspace for both directions of every problem
 * (allocated for B columns on first use and grown for larger B).  A tile that needs an
 * earlier stage waits for it on the device; every wait is bounded by wait_ms (from the
 * CTA's start): past it the kernel records TF_ETIMEOUT in a status word and all CTAs
 * return, leaving the outputs incomplete.  gate, if not NULL, is a DEVICE int that must
 * become nonzero before any tile starts (a start signal from elsewhere; it waits under the
 * same bound).  With use_graph the zeroing of the control words and the launch are
 * recorded once as a CUDA graph and replayed while the key (B, pointers, operator set-ups,
 * options) is unchanged.  The call synchronises `stream` to read the status.
 * Errors: TF_EINVAL (mixed dtypes, bad options, a tile pair not compiled: FP32 8x8,
 * 16x8, 8x4, 4x8; FP64 4x4, 8x8), TF_ETIMEOUT, TF_ENOMEM, TF_ECUDA. */
typedef struct {
  int rows_tile, cols_tile; /* sequence pairs / k1 columns per tile; 0: 8x8 (FP32), 4x4 (FP64) */
  int claim;                /* tiles a CTA claims at once (0: 2)                              */
  double wait_ms;           /* bound of every device-side wait (<= 0: 2000 ms)                */
  const int* gate;          /* DEVICE start gate or NULL                                       */
  int use_graph;            /* record once and replay                                          */
} tf_batch_opts;
tf_status tf_batch_persistent(tf_batch* batch, int64_t B, const void* const* X, void* const* D,
                              const void* const* Y, void* const* XT, const tf_batch_opts* opts,
                              tf_stream stream);

/* Radix order of the generic engine's plan along x (axis 0, length n1) or y (axis 1,
 * length n2): radices from {2, 3, 4, 5, 7, 8} whose product is the length, applied in the
 * given order (each order is a different Stockham pass sequence with its own twiddle
 * table, same transform).  Used by the generic engine (tf_set_engine(op, 1), lengths
 * without a compiled plan, tf_matvec_noalloc and the persistent batch); the compiled
 * plans keep their own.  Waits for the device to be idle.  Errors: TF_EINVAL (axis,
 * radices, product), TF_ENOMEM, TF_ECUDA.  tf_get_radices writes the current order
 * (up to 16 entries) and its length. */
tf_status tf_set_radices(tf_op* op, int axis, const int* radices, int count);
tf_status tf_get_radices(const tf_op* op, int axis, int* radices, int* count);

/* Host helpers of the projected solves (no GPU involved; exported for tests).
 *
 * tf_tridiag_eig_first: eigenvalues of the symmetric tridiagonal matrix with diagonal
 * d[0..n) and off-diagonal e[0..n-1) (e[i] couples i and i+1), by the implicit QL
 * iteration with Wilkinson shifts, together with the first component of each unit
 * eigenvector (the Golub-Welsch weights' square roots, up to sign).  Overwrites d with
 * the eigenvalues (unordered) and writes first[0..n); e is destroyed (needs n entries).
 * An off-diagonal entry counts as zero below eps times its diagonal neighbours or eps
 * times the matrix's infinity norm (eigenvalues to absolute accuracy eps ||T||).  The GKB
 * driver applies it to the Golub-Kahan form of B (zero diagonal, off-diagonal gam_0,
 * bet_0, gam_1, bet_1, ...), whose positive eigenvalues are the singular values s_i and
 * whose eigenvectors' first components are the first row of U over sqrt(2) (Alg. 1).
 * Errors: TF_EINVAL, TF_ENOTCONV.
 *
 * tf_damped_bidiag_solve: y = argmin ||[B; alpha I] y - [b0 e_1; 0]|| for the lower
 * bidiagonal (tp+1) x tp matrix B with diagonal gam[0..tp) and subdiagonal bet[0..tp)
 * (B(j+1, j) = bet[j]), by Givens QR (the Tikhonov-filtered solution of Alg. 1 on all t_p
 * terms).  Errors: TF_EINVAL. */
tf_status tf_tridiag_eig_first(int n, double* d, double* e, double* first);
tf_status tf_damped_bidiag_solve(int tp, const double* gam, const double* bet, double alpha,
                                 double b0, double* y);

/* Message of the calling thread's last failure ("" if none). */
const char* tf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TF_H */
