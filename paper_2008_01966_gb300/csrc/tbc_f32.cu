// FP32 instantiation of the aperture operator (inner iterations of the mixed
// precision solve); compiled separately so that the per-size pass kernels of
// the two precisions build in parallel.
#include "tbc_apply.cuh"

template cavity_status launch_apply<float>(cavity_ctx*, int, const float2*, float2*, void*,
                                          long long);
