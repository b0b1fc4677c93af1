// Mixed-precision stage kernels with the local Lax-Friedrichs split on every
// characteristic field (MRB_FLUX_LLF), one per non-learned reconstruction.
// Same build flags as kern_f32.cu; a separate unit so the variants compile in
// parallel.
#include "mr.cuh"
#include "stage_f32.cuh"

namespace mrb {

void launch_rhs_rk_f32_llf(const Topo& t, const Phys& p, const Pool& pool, int cur, int stage, const double* dt,
                           double* rhs_out, cudaStream_t st, int level) {
  if (p.recon == 2) launch_stage_f32<8 + 2>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.recon == 3) launch_stage_f32<8 + 4>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else if (p.recon == 4) launch_stage_f32<8 + 5>(t, p, pool, cur, stage, dt, rhs_out, st, level);
  else launch_stage_f32<8 + 0>(t, p, pool, cur, stage, dt, rhs_out, st, level);
}

}  // namespace mrb
