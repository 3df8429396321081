// Kernels and launchers for one storage type (float).
#include "ops_impl.cuh"

template struct wd::Ops<float>;
