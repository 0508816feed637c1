// Single-precision instances of the ik-differentiation scale and the plain-window gather.
#include "se_plain.cuh"
namespace se {
SE_PLAIN_INSTANTIATE(float)
}
