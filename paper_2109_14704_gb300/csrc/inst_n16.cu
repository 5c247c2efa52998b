// inst_n16.cu -- kernels for N = 2^16; transform shapes: 2^13 words/CTA x 2^4 words/thread, 2^13 words/CTA x 2^3 words/thread.
#include "inst.cuh"

#define HE_SHAPES_16 {{13, 4}, {13, 3}}
namespace he {
HE_DEGREE(16, 13, 4, HE_SHAPES_16, HE_SHAPE_FN(16, 13, 4) HE_SHAPE_FN(16, 13, 3))
}  // namespace he

HE_DEFINE_DEGREE_OPS(16)
