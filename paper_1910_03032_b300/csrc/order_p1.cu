// Kernels of the order-1 operator (q = 2 and 3).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(1)
