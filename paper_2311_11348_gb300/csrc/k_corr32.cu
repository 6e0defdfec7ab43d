// FP32 instantiation of the correction kernels (mixed-precision mode).
#define CORR_T float
#define CORR_NS corr32
#include "k_corr_impl.cuh"
