// Kernel instantiation for the bf16 storage format (S = __nv_bfloat16, compute in float).
#include "kernels.cuh"

const cslbm_ops cslbm_ops_bf16 = cslbm::Launch<__nv_bfloat16, float>::ops();
