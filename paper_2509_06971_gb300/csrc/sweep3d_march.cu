// sweep3d_march.cu -- placeholder translation unit for the z-marching 3D sweep.
#include "petto_internal.cuh"
