// Kernels of the order-8 operator (q = 9 and 10).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(8)
