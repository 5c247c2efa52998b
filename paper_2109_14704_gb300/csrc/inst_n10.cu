// inst_n10.cu -- kernels for N = 2^10; transform shapes: 2^10 words/CTA x 2^4 words/thread, 2^10 words/CTA x 2^3 words/thread.
#include "inst.cuh"

#define HE_SHAPES_10 {{10, 4}, {10, 3}}
namespace he {
HE_DEGREE(10, 10, 4, HE_SHAPES_10, HE_SHAPE_FN(10, 10, 4) HE_SHAPE_FN(10, 10, 3))
}  // namespace he

HE_DEFINE_DEGREE_OPS(10)
