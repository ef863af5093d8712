// Pass kernels of the pair-of-FP32 operator for log2 sizes 2, 3, 4 (launched from
// tbc_df.cu; one unit per group so that they compile in parallel).
#include "df64.cuh"
#include "tbc_apply.cuh"

TBC_PASS_KERNELS(, df, 2)
TBC_PASS_KERNELS(, df, 3)
TBC_PASS_KERNELS(, df, 4)
