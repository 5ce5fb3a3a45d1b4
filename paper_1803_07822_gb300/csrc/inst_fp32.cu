// Kernel instantiation for the fp32 storage format (S = float, compute in float).
#include "kernels.cuh"

const cslbm_ops cslbm_ops_fp32 = cslbm::Launch<float, float>::ops();
