// fit_disp.cu -- every kernel launch of the library for uint16 raw disparity
// (one translation unit per depth encoding, so the kernels compile in parallel).
#include "sf_launch.cuh"

SF_DEFINE_LAUNCHERS(disp, SF_DEPTH_DISPARITY_U16)
