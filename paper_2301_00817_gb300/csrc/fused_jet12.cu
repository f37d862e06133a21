// fused_jet12.cu -- the fused stage kernel's instantiations with PM = 12
// (fused_kernel.cuh), in a translation unit of their own so that the build
// compiles them in parallel with the others.  Built with approximate FP32
// division and square root.
#include "fused_kernel.cuh"

namespace lesjet {

void launch_stage_jet12(int mode, bool local, bool axis, bool dyn, const FusedGeom& G,
                        const Consts<float>& K, const FusedPtrs& P, const DevScalars* sc,
                        double alpha, const Launch& L) {
  if (dyn)  // (not with an axis: rejected at creation)
    launch_stage_dispatch<false, true, 12>(mode, local, G, K, P, sc, alpha, L);
  else if (axis)
    launch_stage_dispatch<true, false, 12>(mode, local, G, K, P, sc, alpha, L);
  else
    launch_stage_dispatch<false, false, 12>(mode, local, G, K, P, sc, alpha, L);
}

}  // namespace lesjet
