// Kernels of the order-3 operator (q = 4 and 5).
#include "hx_element32_mma.cuh"
HX_DEFINE_ORDER(3)
