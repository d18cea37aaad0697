// FP64 Jacobian / LU (plain form).
#define CAMP_LT double
#define CAMP_SUFFIX f64
#include "launch_impl.cuh"
