// ops_f64_euler.cu -- instantiation of the kernels for double bulk arithmetic, 5 variables.
#include "ops_impl.cuh"

namespace amr {
OpsBase* make_ops_f64_euler(const PhysParams& p) { return new Ops<double, 5>(p); }
}  // namespace amr
