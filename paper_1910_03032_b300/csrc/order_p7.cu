// Kernels of the order-7 operator (q = 8 and 9).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(7)
