// Kernels of the order-2 operator (q = 3 and 4).
#include "hx_element32.cuh"
HX_DEFINE_ORDER(2)
