// Single-precision pipeline without cuFFT (kernels in se_fast.cuh).
#include "se_fast_launch.cuh"
