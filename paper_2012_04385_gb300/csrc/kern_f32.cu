// Mixed-precision stage kernel (MRB_FP32_ACC64): reconstruction and fluxes in
// FP32 from the FP64 state; flux differences, the right-hand side and the
// TVD-RK3 update in FP64.  Built with FMA contraction enabled.
#include "rhs.cuh"

namespace mrb {

void launch_rhs_rk_f32(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                       double* rhs_out, cudaStream_t st) {
  launch_rhs_rk_impl<float>(t, p, pool, cur, stage, dt, rhs_out, st);
}

}  // namespace mrb
