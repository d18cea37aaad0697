// FP32 Jacobian / LU (mixed form) for mechanisms with a water parameter.
#define CAMP_LT float
#define CAMP_SUFFIX f32w
#define CAMP_WATER 1
#include "launch_impl.cuh"
