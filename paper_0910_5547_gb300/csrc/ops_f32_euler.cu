// ops_f32_euler.cu -- instantiation of the kernels for float bulk arithmetic, 5 variables.
#include "ops_impl.cuh"

namespace amr {
OpsBase* make_ops_f32_euler(const PhysParams& p) { return new Ops<float, 5>(p); }
}  // namespace amr
