// Stress kernel (S1 + S2) instantiated for float; the kernel is in k_stress.cuh.
#include "k_stress.cuh"

namespace evp {

template cudaError_t launch_stress<float>(const Geo<float>&, const ModelConst&, const StressArgs<float>&,
                                        cudaStream_t, const TimingHook&);

}  // namespace evp
