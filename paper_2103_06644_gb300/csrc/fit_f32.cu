// fit_f32.cu -- every kernel launch of the library for float32 depth in metres
// (one translation unit per depth encoding, so the kernels compile in parallel).
#include "sf_launch.cuh"

SF_DEFINE_LAUNCHERS(f32, SF_DEPTH_F32)
