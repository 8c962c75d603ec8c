// echo_kernels_flat.cu -- instantiation of the metric-dependent kernels for
// the flat (Minkowski, Cartesian) metric.
#include "echo_kernels.cuh"
#define ECHO_MK 0
#include "echo_launch_mk.inc"
