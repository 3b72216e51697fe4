// complex-FP64 instantiation of the FFT matvec (see matvec_impl.cuh)
#include "matvec_impl.cuh"

namespace vie {
template vie_status matvec<double2>(vie_plan_s*, const double2*, double2*, const double2*, const double2*,
                                    double2*, double2*, cudaStream_t);
template vie_status xpass<double2>(vie_plan_s*, const double2*, double2*, double2*, int, cudaStream_t);
}  // namespace vie
