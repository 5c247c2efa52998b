// inst_n16.cu -- kernels for N = 2^16; transform shapes: 2^13 words/CTA x 2^4 words/thread (default), 2^13 x 2^3, 2^12 x 2^4 (clusters of 16, the non-portable size: measured 13 % faster forward).
#include "inst.cuh"

#define HE_SHAPES_16 {{13, 4}, {13, 3}, {12, 4}}
namespace he {
HE_DEGREE(16, 13, 4, HE_SHAPES_16, HE_SHAPE_FN(16, 13, 4) HE_SHAPE_FN(16, 13, 3) HE_SHAPE_FN(16, 12, 4))
}  // namespace he

HE_DEFINE_DEGREE_OPS(16)
