// ops_f64_mhd.cu -- instantiation of the kernels for double bulk arithmetic, 9 variables.
#include "ops_impl.cuh"

namespace amr {
OpsBase* make_ops_f64_mhd(const PhysParams& p) { return new Ops<double, 9>(p); }
}  // namespace amr
