// inst_n15.cu -- kernels for N = 2^15; transform shapes: 2^12 words/CTA x 2^4 words/thread, 2^13 words/CTA x 2^4 words/thread, 2^12 words/CTA x 2^3 words/thread, 2^13 words/CTA x 2^3 words/thread, and the 2^12-word shapes at 3 and 2 CTAs per SM.
#include "inst.cuh"

// (the last two: the 2^12-word shapes compiled for 3 and 2 CTAs per SM, i.e.
// 85 and 64 registers a thread instead of 64 and 42)
#define HE_SHAPES_15 {{12, 4}, {13, 4}, {12, 3}, {13, 3}, {12, 4 | 3 << 4}, {12, 3 | 2 << 4}}
namespace he {
HE_DEGREE(15, 12, 4, HE_SHAPES_15, HE_SHAPE_FN(15, 12, 4) HE_SHAPE_FN(15, 13, 4) HE_SHAPE_FN(15, 12, 3) HE_SHAPE_FN(15, 13, 3)
          HE_SHAPE_FN_OCC(15, 12, 4, 3) HE_SHAPE_FN_OCC(15, 12, 3, 2))
}  // namespace he

HE_DEFINE_DEGREE_OPS(15)
