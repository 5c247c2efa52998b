// inst_n12.cu -- kernels for N = 2^12; transform shapes: 2^12 words/CTA x 2^4 words/thread, 2^12 words/CTA x 2^3 words/thread, 2^11 words/CTA x 2^4 words/thread, 2^10 words/CTA x 2^4 words/thread.
#include "inst.cuh"

#define HE_SHAPES_12 {{12, 4}, {12, 3}, {11, 4}, {10, 4}}
namespace he {
HE_DEGREE(12, 12, 4, HE_SHAPES_12, HE_SHAPE_FN(12, 12, 4) HE_SHAPE_FN(12, 12, 3) HE_SHAPE_FN(12, 11, 4) HE_SHAPE_FN(12, 10, 4))
}  // namespace he

HE_DEFINE_DEGREE_OPS(12)
