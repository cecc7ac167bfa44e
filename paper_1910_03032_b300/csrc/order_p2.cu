// Kernels of the order-2 operator (q = 3 and 4).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(2)
