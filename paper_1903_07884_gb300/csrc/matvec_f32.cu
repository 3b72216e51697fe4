// complex-FP32 instantiation of the FFT matvec (see matvec_impl.cuh)
#include "matvec_impl.cuh"

namespace vie {
template vie_status matvec<float2>(vie_plan_s*, const float2*, float2*, const float2*, const float2*, float2*,
                                   float2*, cudaStream_t);
template vie_status xpass<float2>(vie_plan_s*, const float2*, float2*, float2*, int, cudaStream_t);
}  // namespace vie
