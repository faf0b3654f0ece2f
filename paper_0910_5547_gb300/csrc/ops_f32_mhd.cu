// ops_f32_mhd.cu -- instantiation of the kernels for float bulk arithmetic, 9 variables.
#include "ops_impl.cuh"

namespace amr {
OpsBase* make_ops_f32_mhd(const PhysParams& p) { return new Ops<float, 9>(p); }
}  // namespace amr
