// Pass kernels of the pair-of-FP32 operator for log2 sizes 9 (launched from
// tbc_df.cu; one unit per group so that they compile in parallel).
#include "df64.cuh"
#include "tbc_apply.cuh"

TBC_PASS_KERNELS(, df, 9)
