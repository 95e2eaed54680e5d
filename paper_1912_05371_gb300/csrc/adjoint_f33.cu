// The discrete adjoint's kernels and launchers for float fields in blocks of 33^3.
#include "adjoint_kernels.cuh"

ACM_ADJ_INSTANTIATE(float, 33)
