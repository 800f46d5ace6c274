// Stress kernel (S1 + S2) instantiated for float; the kernel is in k_stress.cuh.
#include "k_stress.cuh"

namespace evp {

template cudaError_t launch_stress<float>(const Geo<float>&, const ModelConst&, const StressArgs<float>&,
                                        cudaStream_t, const TimingHook&);
template cudaError_t launch_stress_batch<float>(const StressBatch<float>&, int, int, bool, const int4*, int, int,
                                               cudaStream_t);
template int stress_ctas_per_sm<float>();

int stress_tile_x() { return TX; }
int stress_tile_y() { return TY; }

}  // namespace evp
