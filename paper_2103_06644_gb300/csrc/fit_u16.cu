// fit_u16.cu -- every kernel launch of the library for uint16 depth in raw units
// (one translation unit per depth encoding, so the kernels compile in parallel).
#include "sf_launch.cuh"

SF_DEFINE_LAUNCHERS(u16, SF_DEPTH_U16)
