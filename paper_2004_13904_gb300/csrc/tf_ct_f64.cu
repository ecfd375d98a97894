// Compile-time-plan product kernels, double instantiations (see tf_ct_kernels.cuh).
#include "tf_ct_kernels.cuh"

namespace tfk {
TF_DEFINE_OOB_READER(oob_read_ct_f64)
TF_CT_DEFINE_DISPATCH(double, TF_CT_MENU)
}  // namespace tfk
