// Internal launchers shared by the C-ABI layer and the kernels (not part of the ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "tf_check.cuh"
#include "tf_fft.cuh"

namespace tfk {

// Rows stage, real -> half spectrum (App. A: 1-D FFTs along x of the embedded rows).
// Row rho of column b holds row_len reals at src + b*src_ld + rho*row_len; they are
// scaled by scale[rho*row_len + n] (if non-null), placed at [seq_off, seq_off+row_len)
// of a zero sequence of length plan.n, transformed, and the nh = n/2+1 outputs are
// written to dst + b*dst_ld + rho*hs (hs >= nh: the row stride of half-spectrum
// buffers).  Two rows share one complex transform.
template <typename T> struct RowsR2C {
  const T* src; int64_t src_ld; int row_len; int nrows; int seq_off; const T* scale;
  typename CT<T>::C* dst; int64_t dst_ld; int nh; int hs;
  FftPlan plan; const typename CT<T>::C* tw;
};

// Rows stage, half spectrum -> real window: inverse of the above; outputs sequence
// entries [seq_off, seq_off+out_len) times scale[rho*out_len + i] to dst.
template <typename T> struct RowsC2R {
  const typename CT<T>::C* src; int64_t src_ld; int nh; int hs; int nrows;
  T* dst; int64_t dst_ld; int out_len; int seq_off; const T* scale;
  FftPlan plan; const typename CT<T>::C* tw;
};

// Column stage of G x: for each k1 column, FFT along y of every layer's rows,
// multiply-accumulate with the layer spectra (sum over layers in the frequency domain),
// inverse FFT, keep rows [ny-1, ny-1+sy).  Rows of nh values with row stride hs.
template <typename T> struct ColsFwd {
  const typename CT<T>::C* z; int64_t z_ld;       // [nz*ny][hs] per column
  const typename CT<T>::C* spec;                  // [nz][n2][hs]
  typename CT<T>::C* s; int64_t s_ld;             // [sy][hs] per column
  int nh, hs, ny, sy, nz;
  FftPlan plan; const typename CT<T>::C* tw;
  int ncols;                                      // columns of the launch (set by the launcher)
};

// Column stage of G^T y: FFT along y of the data rows placed at [ny-1, ny-1+sy), then
// per layer multiply by the conjugate spectrum, inverse FFT, keep rows [0, ny).
template <typename T> struct ColsAdj {
  const typename CT<T>::C* z; int64_t z_ld;       // [sy][hs] per column
  const typename CT<T>::C* spec;                  // [nz][n2][hs]
  typename CT<T>::C* u; int64_t u_ld;             // [nz*ny][hs] per column
  int nh, hs, ny, sy, nz;
  FftPlan plan; const typename CT<T>::C* tw;
};

// ---- persistent batch kernel (tf_batch_kernels.cu) ----------------------------------
//
// One launch runs the generic engine's product stages of many problems.  The work items
// are tiles of columns; a segment is one stage of one problem and direction, a
// contiguous range of items (column-major: item = first + col * tiles + tile).  Items
// are claimed in increasing order, and a stage's items come after those of the stage it
// waits on, so every wait is for items already claimed by running CTAs.
struct BatchSeg {
  long long first;   // first work item of the segment
  int kind;          // 0 rows_r2c, 1 cols_fwd, 2 rows_c2r, 3 cols_adj
  int tiles;         // tiles per column
  int cols;          // columns
  int args;          // index of the stage's arguments
  int wait;          // counters (one per column) of the stage this one needs, -1 if none
  int wait_target;   // tiles per column of that stage
  int count;         // counters (one per column) this stage's finished tiles add to
};
template <typename T> union BatchArgs {
  RowsR2C<T> r2c;
  ColsFwd<T> fwd;
  RowsC2R<T> c2r;
  ColsAdj<T> adj;
};
struct BatchCtl {
  unsigned long long* work;  // next unclaimed item (zero at launch)
  int* counters;             // finished tiles per (segment, column) (zero at launch)
  int* status;               // 0 at launch; 6 (TF_ETIMEOUT) once a wait ran out
  const int* gate;           // NULL, or: no item starts before *gate != 0
  long long total;           // work items
  int nseg;
  const BatchSeg* seg;       // nseg segments in increasing `first`
  const void* args;          // BatchArgs<T>[]
  unsigned long long budget_ns;  // every wait gives up this long after the CTA started
  int claim;                 // items a CTA claims at once
};
// Launches the persistent kernel with rows tile tb and column tile tk (4, 8 or 16) and
// `smem` bytes of dynamic shared memory (the largest stage's need), one grid of resident
// CTAs; *grid receives its size.
// Returns cudaErrorInvalidValue for a tile pair the dtype was not compiled with (FP32:
// 8x8, 16x8, 8x4, 4x8; FP64: 4x4, 8x8).
template <typename T>
cudaError_t launch_batch(const BatchCtl& c, int tb, int tk, size_t smem, cudaStream_t s, int* grid);
template <> cudaError_t launch_batch<float>(const BatchCtl&, int, int, size_t, cudaStream_t, int*);
template <> cudaError_t launch_batch<double>(const BatchCtl&, int, int, size_t, cudaStream_t, int*);

// The generic engine's six stage arguments of one operator's products on columns of
// X / D / Y / XT (leading dimensions n and m): G X (rows_r2c, cols_fwd, rows_c2r) through
// the workspace columns fw1 / fw2 and G^T Y (rows_r2c, cols_adj, rows_c2r) through aw1 /
// aw2 (workspace column strides as the operator's own workspace).  Defined in tf_api.cu.
template <typename T> struct ProductStages {
  RowsR2C<T> f0; ColsFwd<T> f1; RowsC2R<T> f2;
  RowsR2C<T> a0; ColsAdj<T> a1; RowsC2R<T> a2;
};
struct OpGeneric {
  int dtype;                     // tf_dtype
  int64_t m, n, w1_per_col, w2_per_col;
  size_t csize;
  int n1, n2, tw1, tw2, rows_model, rows_data, nh;
};

struct TableArgs {
  int kind;                // 0 gravity, 1 magnetic
  int n1min, n2min, nz, nx, ny, pxl, pyl;
  double dx, dy, station_z;
  const double* z_edges;   // device, nz+1
  double fx, fy, fz, field;  // magnetic: field direction and strength (nT)
  double* out;             // [nz][n2min][n1min]
  // Gauss-Legendre rules for cells away from the station (see k_table)
  double g6x[6], g6w[6], g8x[8], g8w[8], g14x[14], g14w[14];
};

struct SpecArgs {
  const double2* ht; int n2min; int nh; int nz; double scale;   // ht: [nz][n2min][nh]
  double2* spec; int hs;   // [nz][n2][hs]
  FftPlan plan; const double2* tw;
};

template <typename T> cudaError_t launch_rows_r2c(const RowsR2C<T>& a, int ncols, int tb, cudaStream_t s);
template <typename T> cudaError_t launch_rows_c2r(const RowsC2R<T>& a, int ncols, int tb, cudaStream_t s);
template <typename T> cudaError_t launch_cols_fwd(const ColsFwd<T>& a, int ncols, int tk, cudaStream_t s);
template <typename T> cudaError_t launch_cols_adj(const ColsAdj<T>& a, int ncols, int tk, cudaStream_t s);
// Loads the generic engine's forward-product kernels (rows_r2c, cols_fwd, rows_c2r) on
// the current device and raises their shared-memory limits for lengths n1 (row
// transforms, tw1 twiddles) and n2 (column transforms), rows tile tb and column tile tk,
// so that later launches of that configuration make no load or attribute call.
template <typename T> cudaError_t prepare_forward_generic(int n1, int tw1, int n2, int tw2, int tb, int tk);
// Compile-time-plan variants of the four product stages (tf_ct_kernels.cuh); they
// return cudaErrorNotSupported, before any CUDA call, for lengths off their menu.
template <typename T> cudaError_t ct_rows_r2c(const RowsR2C<T>& a, int ncols, cudaStream_t s);
template <typename T> cudaError_t ct_rows_c2r(const RowsC2R<T>& a, int ncols, cudaStream_t s);
template <typename T> cudaError_t ct_cols_fwd(const ColsFwd<T>& a, int ncols, cudaStream_t s);
template <typename T> cudaError_t ct_cols_adj(const ColsAdj<T>& a, int ncols, cudaStream_t s);
template <> cudaError_t ct_rows_r2c<float>(const RowsR2C<float>&, int, cudaStream_t);
template <> cudaError_t ct_rows_r2c<double>(const RowsR2C<double>&, int, cudaStream_t);
template <> cudaError_t ct_rows_c2r<float>(const RowsC2R<float>&, int, cudaStream_t);
template <> cudaError_t ct_rows_c2r<double>(const RowsC2R<double>&, int, cudaStream_t);
template <> cudaError_t ct_cols_fwd<float>(const ColsFwd<float>&, int, cudaStream_t);
template <> cudaError_t ct_cols_fwd<double>(const ColsFwd<double>&, int, cudaStream_t);
template <> cudaError_t ct_cols_adj<float>(const ColsAdj<float>&, int, cudaStream_t);
template <> cudaError_t ct_cols_adj<double>(const ColsAdj<double>&, int, cudaStream_t);
// Status word of the persistent bulk-copy row kernels: TF_ETIMEOUT (6) once a bounded wait
// ran out, else 0; `clear` resets it.
unsigned ct_pipe_status(bool clear);
// Transform lengths that have compile-time plans (ascending), with their radix lists.
int ct_menu_count();
int ct_menu_length(int i);
int ct_menu_radices(int i, int* radices /* up to kMaxPass */);
// radix list of the single-precision column kernels' plan for length n (0 when n has none)
int ct_menu_cols_radices(int n, int* radices /* up to kMaxPass */);

// Bounds-check records of each kernel translation unit (false in unchecked builds).
bool oob_read_generic(OobRecord* out, bool clear);
bool oob_read_ct_f32(OobRecord* out, bool clear);
bool oob_read_ct_f64(OobRecord* out, bool clear);
bool oob_read_batch_f32(OobRecord* out, bool clear);
bool oob_read_batch_f64(OobRecord* out, bool clear);

cudaError_t launch_table(const TableArgs& a, cudaStream_t s);
// Re-orthogonalisation helpers on a stack of k vectors A[j*lda + i] (dtype 0: float,
// 1: double), FP64 accumulation.
cudaError_t launch_rows_dot(int dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                            const void* x, double* y, cudaStream_t s);
cudaError_t launch_rows_axpy(int dtype, const void* A, int64_t lda, int64_t k, int64_t len,
                             const double* c, void* x, cudaStream_t s);
// FMA-chain probe: two timed launches of `blocks` x 256 threads, 8 chains x iters each.
cudaError_t launch_fma_probe(int dtype, void* out, int blocks, int iters, float* ms, cudaStream_t s);
cudaError_t launch_spectrum(const SpecArgs& a, int tk, cudaStream_t s);
cudaError_t launch_to_f32(const double2* src, float2* dst, int64_t count, cudaStream_t s);

size_t smem_rows(int n, int tw_count, int tb, size_t csize);
size_t smem_cols(int n, int tw_count, int tk, size_t csize);

}  // namespace tfk
