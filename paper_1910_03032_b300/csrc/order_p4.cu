// Kernels of the order-4 operator (q = 5 and 6).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(4)
