// Internal hooks of tf_api.cu used by the IRLS drivers (tf_irls.cu); not part of the ABI.
#pragma once
#include <stdint.h>

#include <vector>

#include "../../include/tf.h"

namespace tfk {

struct OpInfo {
  tf_dtype dtype;
  int64_t m, n;
  int nx, ny, nz;
  std::vector<double> z_edges;  // nz + 1, z positive down
  double station_z;
  int device;
};

// The operator's sizes and geometry.
tf_status op_info(const tf_op* op, OpInfo* out);
// Identity of the operator's launch configuration: its workspace address and column
// chunk, its engine and tiles (a CUDA graph of its products is valid while these hold).
struct OpLaunchKey {
  const void* w1;
  int64_t chunk;
  int engine, rows_tile, cols_tile;
  const void *tw1, *tw2;   // the generic plans' twiddle tables (replaced by tf_set_radices)
  bool operator==(const OpLaunchKey& o) const {
    return w1 == o.w1 && chunk == o.chunk && engine == o.engine && rows_tile == o.rows_tile &&
           cols_tile == o.cols_tile && tw1 == o.tw1 && tw2 == o.tw2;
  }
};
OpLaunchKey op_launch_key(const tf_op* op);
// Sizes of the operator's generic-engine stages (for the persistent batch kernel).
struct OpGeneric;
OpGeneric op_generic(const tf_op* op);
template <typename T> struct ProductStages;
template <typename T>
void op_product_stages(const tf_op* op, const T* X, T* D, const T* Y, T* XT, void* fw1, void* fw2,
                       void* aw1, void* aw2, ProductStages<T>* out);
// Sets the calling thread's last-error message (what tf_last_error returns) and returns st.
tf_status api_fail(tf_status st, const char* fmt, ...);

}  // namespace tfk
