// Kernel instantiation for the fp16 storage format (S = __half, compute in float).
#include "kernels.cuh"

const cslbm_ops cslbm_ops_fp16 = cslbm::Launch<__half, float>::ops();
