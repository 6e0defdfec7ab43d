// FP64 instantiation of the correction kernels.
#define CORR_T double
#define CORR_NS corr64
#include "k_corr_impl.cuh"
