// inst_n11.cu -- kernels for N = 2^11; transform shapes: 2^11 words/CTA x 2^4 words/thread, 2^11 words/CTA x 2^3 words/thread, 2^10 words/CTA x 2^4 words/thread.
#include "inst.cuh"

#define HE_SHAPES_11 {{11, 4}, {11, 3}, {10, 4}}
namespace he {
HE_DEGREE(11, 11, 4, HE_SHAPES_11, HE_SHAPE_FN(11, 11, 4) HE_SHAPE_FN(11, 11, 3) HE_SHAPE_FN(11, 10, 4))
}  // namespace he

HE_DEFINE_DEGREE_OPS(11)
