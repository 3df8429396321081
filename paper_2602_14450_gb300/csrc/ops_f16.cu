// Kernels and launchers for one storage type (__half).
#include "ops_impl.cuh"

template struct wd::Ops<__half>;
