// FP32 Jacobian / LU (mixed form).
#define CAMP_LT float
#define CAMP_SUFFIX f32
#include "launch_impl.cuh"
