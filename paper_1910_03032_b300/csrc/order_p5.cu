// Kernels of the order-5 operator (q = 6 and 7).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(5)
