// vlb_step16.cu -- time-step launches for populations stored in 16 bits
// (IEEE half, bfloat16) with FP32 arithmetic.
#include "vlb_step.cuh"

namespace vlb {

cudaError_t launch_step_16(const vlb_sim *sim, int odd, cudaStream_t s) {
  const int q = sim->mesh->md.q;
  if (sim->p.precision == VLB_BF16)
    return q == 9 ? launch_step_t<9, __nv_bfloat16, float>(sim, odd, s)
                  : launch_step_t<19, __nv_bfloat16, float>(sim, odd, s);
  return q == 9 ? launch_step_t<9, __half, float>(sim, odd, s) : launch_step_t<19, __half, float>(sim, odd, s);
}

}  // namespace vlb
