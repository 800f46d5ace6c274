// Stress kernel (S1 + S2) instantiated for double; the kernel is in k_stress.cuh.
#include "k_stress.cuh"

namespace evp {

template cudaError_t launch_stress<double>(const Geo<double>&, const ModelConst&, const StressArgs<double>&,
                                        cudaStream_t, const TimingHook&);
template cudaError_t launch_stress_batch<double>(const StressBatch<double>&, int, int, bool, const int4*, int, int,
                                               cudaStream_t);
template int stress_ctas_per_sm<double>();

}  // namespace evp
