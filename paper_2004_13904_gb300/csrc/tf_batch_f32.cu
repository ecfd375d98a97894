// Persistent batch kernel instantiated for float data (tile pairs rows x columns:
// 8 x 8, 16 x 8, 8 x 4, 4 x 8).
#include "tf_batch_kernels.cuh"

namespace tfk {

template <>
cudaError_t launch_batch<float>(const BatchCtl& c, int tb, int tk, size_t smem, cudaStream_t s,
                            int* grid) {
  typedef float T;
  switch (tb * 100 + tk) {
    TF_BATCH_CASE(8, 8)
    TF_BATCH_CASE(16, 8)
    TF_BATCH_CASE(8, 4)
    TF_BATCH_CASE(4, 8)
    default: return cudaErrorInvalidValue;
  }
}

TF_DEFINE_OOB_READER(oob_read_batch_f32)

}  // namespace tfk
