// Stress kernel (S1 + S2) instantiated for double; the kernel is in k_stress.cuh.
#include "k_stress.cuh"

namespace evp {

template cudaError_t launch_stress<double>(const Geo<double>&, const ModelConst&, const StressArgs<double>&,
                                        cudaStream_t, const TimingHook&);

}  // namespace evp
