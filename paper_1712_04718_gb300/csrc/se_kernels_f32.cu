// Single-precision instances of the SE kernels.
#include "se_launch.cuh"
namespace se {
SE_INSTANTIATE(float)
}
