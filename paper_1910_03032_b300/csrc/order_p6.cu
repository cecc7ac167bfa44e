// Kernels of the order-6 operator (q = 7 and 8).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(6)
