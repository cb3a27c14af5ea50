// Row kernels and binning for the plus-times fp32 semiring.
#include <algorithm>
#define MSG_CAT2(a, b) a##b
#define MSG_CAT(a, b) MSG_CAT2(a, b)
#define MSG_SR MSGEMM_PLUS_TIMES_F32
#define MSG_SUFFIX f32
#include "rows_inst.cuh"
