// Kernel instantiation for the fp64 storage format (S = double, compute in double).
#include "kernels.cuh"

const cslbm_ops cslbm_ops_fp64 = cslbm::Launch<double, double>::ops();
