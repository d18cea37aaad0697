// FP64 Jacobian / LU (plain form) for mechanisms with a water parameter.
#define CAMP_LT double
#define CAMP_SUFFIX f64w
#define CAMP_WATER 1
#include "launch_impl.cuh"
