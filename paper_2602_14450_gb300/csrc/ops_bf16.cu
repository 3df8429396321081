// Kernels and launchers for one storage type (__nv_bfloat16).
#include "ops_impl.cuh"

template struct wd::Ops<__nv_bfloat16>;
