// The discrete adjoint's kernels and launchers for double fields in blocks of 9^3.
#include "adjoint_kernels.cuh"

ACM_ADJ_INSTANTIATE(double, 9)
