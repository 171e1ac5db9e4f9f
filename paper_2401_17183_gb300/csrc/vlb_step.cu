// vlb_step.cu -- time-step launches for FP64 and FP32 populations, and the
// dispatch over storage types (the 16-bit kernels are compiled in
// vlb_step16.cu).
#include "vlb_step.cuh"

namespace vlb {

cudaError_t launch_step_16(const vlb_sim *sim, int odd, cudaStream_t s);

cudaError_t launch_step(const vlb_sim *sim, int odd, cudaStream_t s) {
  const int q = sim->mesh->md.q;
  switch (sim->p.precision) {
    case VLB_F64:
      return q == 9 ? launch_step_t<9, double, double>(sim, odd, s)
                    : launch_step_t<19, double, double>(sim, odd, s);
    case VLB_F32:
      return q == 9 ? launch_step_t<9, float, float>(sim, odd, s)
                    : launch_step_t<19, float, float>(sim, odd, s);
    default:
      return launch_step_16(sim, odd, s);
  }
}

}  // namespace vlb
