/*
 * A plain C caller of libtf.so (include/tf.h): builds a gravity operator, applies G and
 * G^T to device vectors with the CUDA runtime for memory, and prints the results, one
 * value per line (%.17g), so that a test can compare them with the Python binding's.
 *
 * Usage: products <sx> <sy> <nz> <pad> <f32|f64>
 * Geometry: pad cells on every side, 50 m cells, layer r spans [50 r, 50 (r+1)] m,
 * stations at depth 0.  Inputs: x_i = sin(0.37 i) + 0.25, y_j = cos(0.11 j).
 * Output: "m n", then the m values of G x, then the n values of G^T y.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include "tf.h"

static int fail(const char* what) {
  fprintf(stderr, "%s: %s\n", what, tf_last_error());
  return 1;
}

int main(int argc, char** argv) {
  if (argc != 6) {
    fprintf(stderr, "usage: %s sx sy nz pad f32|f64\n", argv[0]);
    return 2;
  }
  const int sx = atoi(argv[1]), sy = atoi(argv[2]), nz = atoi(argv[3]), pad = atoi(argv[4]);
  const tf_dtype dt = strcmp(argv[5], "f32") == 0 ? TF_F32 : TF_F64;
  const size_t es = dt == TF_F32 ? sizeof(float) : sizeof(double);
  double* z = (double*)malloc(sizeof(double) * (size_t)(nz + 1));
  for (int r = 0; r <= nz; ++r) z[r] = 50.0 * r;
  tf_grid g;
  g.sx = sx; g.sy = sy; g.nz = nz;
  g.pxl = g.pxr = g.pyl = g.pyr = pad;
  g.dx = g.dy = 50.0;
  g.z_edges = z;
  g.station_z = 0.0;

  tf_op* op = NULL;
  if (tf_create_gravity(&g, dt, NULL, &op) != TF_OK) return fail("tf_create_gravity");
  int64_t m = 0, n = 0;
  if (tf_dims(op, &m, &n) != TF_OK) return fail("tf_dims");

  void* hx = malloc(es * (size_t)n);
  void* hy = malloc(es * (size_t)m);
  for (int64_t i = 0; i < n; ++i) {
    const double v = sin(0.37 * (double)i) + 0.25;
    if (dt == TF_F32) ((float*)hx)[i] = (float)v; else ((double*)hx)[i] = v;
  }
  for (int64_t j = 0; j < m; ++j) {
    const double v = cos(0.11 * (double)j);
    if (dt == TF_F32) ((float*)hy)[j] = (float)v; else ((double*)hy)[j] = v;
  }
  void *dx = NULL, *dy = NULL, *dd = NULL, *dxt = NULL;
  if (cudaMalloc(&dx, es * (size_t)n) != cudaSuccess || cudaMalloc(&dy, es * (size_t)m) != cudaSuccess ||
      cudaMalloc(&dd, es * (size_t)m) != cudaSuccess || cudaMalloc(&dxt, es * (size_t)n) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  cudaMemcpy(dx, hx, es * (size_t)n, cudaMemcpyHostToDevice);
  cudaMemcpy(dy, hy, es * (size_t)m, cudaMemcpyHostToDevice);
  if (tf_matvec(op, dx, dd, NULL, NULL, NULL) != TF_OK) return fail("tf_matvec");
  if (tf_rmatvec(op, dy, dxt, NULL, NULL, NULL) != TF_OK) return fail("tf_rmatvec");
  if (cudaDeviceSynchronize() != cudaSuccess) {
    fprintf(stderr, "device error: %s\n", cudaGetErrorString(cudaGetLastError()));
    return 1;
  }
  cudaMemcpy(hy, dd, es * (size_t)m, cudaMemcpyDeviceToHost);
  cudaMemcpy(hx, dxt, es * (size_t)n, cudaMemcpyDeviceToHost);
  printf("%lld %lld\n", (long long)m, (long long)n);
  for (int64_t j = 0; j < m; ++j)
    printf("%.17g\n", dt == TF_F32 ? (double)((float*)hy)[j] : ((double*)hy)[j]);
  for (int64_t i = 0; i < n; ++i)
    printf("%.17g\n", dt == TF_F32 ? (double)((float*)hx)[i] : ((double*)hx)[i]);

  cudaFree(dx); cudaFree(dy); cudaFree(dd); cudaFree(dxt);
  free(hx); free(hy); free(z);
  if (tf_destroy(op) != TF_OK) return fail("tf_destroy");
  return 0;
}
