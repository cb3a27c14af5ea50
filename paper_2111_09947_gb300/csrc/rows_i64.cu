// Row kernels and binning for the plus-times int64 semiring.
#include <algorithm>
#define MSG_CAT2(a, b) a##b
#define MSG_CAT(a, b) MSG_CAT2(a, b)
#define MSG_SR MSGEMM_PLUS_TIMES_I64
#define MSG_SUFFIX i64
#include "rows_inst.cuh"
