// Kernels and launchers for one storage type (double).
#include "ops_impl.cuh"

template struct wd::Ops<double>;
