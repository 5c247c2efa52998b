// ntt_core.cuh -- block-level negacyclic NTT building blocks for sm_103a.
//
// One limb of N = B * C words is transformed by a thread-block cluster of C
// CTAs; CTA m owns the contiguous block [m B, (m + 1) B) of positions in
// shared memory (B = 2^LOG_B words, 16 per thread).
//
// Forward transform (Sec. II-B with the psi twist folded into bit-reversed
// twiddles; Cooley-Tukey stages with Harvey's lazy butterfly, Algorithm 1):
//   stage S (0 .. log N - 1) has 2^S groups of 2 N / 2^S positions; group g
//   uses W = psi^brv(2^S + g) and pairs positions j and j + N / 2^(S+1).
//   * The first log C stages pair positions in different CTAs. Each thread
//     loads whole columns {t B + j : t < C} from global memory, runs the
//     radix-C network in registers and scatters element t to CTA t through
//     distributed shared memory (st.shared::cluster). This is the paper's
//     "global memory" stage group, done without a second pass over HBM.
//   * The remaining log B stages stay inside one CTA: rounds of up to four
//     stages (radix 16) in registers, exchanging through shared memory
//     between rounds (the paper's SLM rounds, Sec. III-B, with a higher
//     radix than its radix-8 because registers are 64-bit pairs here).
//   * The last round reduces from [0, 4p) to [0, p) (the paper's last-round
//     offsetting, fused) and hands each canonical value to the caller's store
//     functor.
// Inverse transform: the mirror image with Gentleman-Sande butterflies on
// [0, 2p); local rounds first, cross-CTA stages last, N^-1 folded into the
// final stage.
//
// Shared-memory layout: element l of the block sits at word
// l ^ ((l >> 4) & 15), which keeps every access pattern below free of bank
// conflicts (each half warp touches 16 distinct 8-byte bank pairs).
#pragma once
#include <stdint.h>

#include <utility>

#include "modarith.cuh"

namespace he {

__device__ __forceinline__ u32 swz(u32 l) { return l ^ ((l >> 4) & 15u); }

__device__ __forceinline__ u32 cluster_ctarank()
{
    u32 r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ u32 smem_u32(const void *p) { return (u32)__cvta_generic_to_shared(p); }

__device__ __forceinline__ u32 map_to_rank(u32 addr, u32 rank)
{
    u32 r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

__device__ __forceinline__ void st_cluster(u32 addr, u64 v)
{
    asm volatile("st.shared::cluster.u64 [%0], %1;" ::"r"(addr), "l"(v) : "memory");
}

__device__ __forceinline__ u64 ld_cluster(u32 addr)
{
    u64 v;
    asm volatile("ld.shared::cluster.u64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
    return v;
}

__device__ __forceinline__ ulonglong2 ld_tw(const ulonglong2 *tw, u32 idx) { return __ldg(tw + idx); }

template <int LOG_B_, int LOG_C_>
struct NttShape {
    static constexpr int LOG_B = LOG_B_;
    static constexpr int LOG_C = LOG_C_;
    static constexpr int LOG_N = LOG_B + LOG_C;
    static constexpr u32 B = 1u << LOG_B;
    static constexpr u32 C = 1u << LOG_C;
    static constexpr u32 N = 1u << LOG_N;
    static constexpr int E = 16;                  // words per thread
    static constexpr u32 T = B / E;               // threads per CTA
    static constexpr int NROUND = (LOG_B + 3) / 4;
    static constexpr int LAST_R = LOG_B - 4 * (NROUND - 1);
    static constexpr u32 SMEM_BYTES = B * 8;
    static_assert(LOG_C <= 3, "portable clusters hold at most 8 CTAs");
    static_assert(LOG_B >= 9, "at least 32 threads per CTA");
};

template <int R_, int S0_, int LOG_B>
struct Round {
    static constexpr int R = R_;                  // stages in this round
    static constexpr int S0 = S0_;                // first local stage
    static constexpr int SUB = 16 >> R;           // subgroups per thread
    static constexpr int LOG_TL = LOG_B - S0 - R; // log of the smallest gap
    static constexpr u32 TL = 1u << LOG_TL;
};

// Block-local position of element u of subgroup i of this thread in a round.
template <class Rd>
__device__ __forceinline__ u32 round_pos(u32 tid, int i, int u)
{
    u32 sg = tid * Rd::SUB + (u32)i;
    u32 k = sg & (Rd::TL - 1);
    u32 g = sg >> Rd::LOG_TL;
    return (g << (Rd::LOG_TL + Rd::R)) + k + (u32)u * Rd::TL;
}

// Barrier between two consecutive block transforms in one CTA: the next
// transform's first writes to shared memory (remote ones for a cluster) must
// not overtake reads of the previous transform.
template <class Sh>
__device__ __forceinline__ void ntt_barrier()
{
    if constexpr (Sh::LOG_C > 0)
        cluster_sync_all();
    else
        __syncthreads();
}

// ---------------------------------------------------------------- forward

// Group base of subgroup i in a round: the index, at the round's first stage,
// of the butterfly group that holds the subgroup. At internal stage q the
// twiddle of the group holding element u is 2^S + (G << q) + (u >> (R - q)),
// because P >> (log N - S) splits into the aligned part of the subgroup's
// base and the top q bits of u.
template <class Sh, class Rd>
__device__ __forceinline__ u32 round_group_base(u32 tid, int i, u32 m)
{
    u32 sg = tid * Rd::SUB + (u32)i;
    u32 g = sg >> Rd::LOG_TL;
    return (m << (Sh::LOG_B - Rd::LOG_TL - Rd::R)) + g;
}

template <class Sh, class Rd, int q>
__device__ __forceinline__ void fwd_stage(u64 (&x)[16], u32 tid, u32 m, const ulonglong2 *tw, u64 p,
                                          u64 two_p)
{
    constexpr int S = Sh::LOG_C + Rd::S0 + q;     // global stage
    constexpr int half = 1 << (Rd::R - 1 - q);
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++) {
        const u32 G = round_group_base<Sh, Rd>(tid, i, m);
#pragma unroll
        for (int grp = 0; grp < (1 << q); grp++) {
            const ulonglong2 w = ld_tw(tw, (1u << S) + (G << q) + (u32)grp);
#pragma unroll
            for (int v = 0; v < half; v++) {
                const int u = grp * 2 * half + v;
                ct_butterfly(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], w.x, w.y, p, two_p);
            }
        }
    }
}

template <class Sh, class Rd, int... Q>
__device__ __forceinline__ void fwd_round_stages(u64 (&x)[16], u32 tid, u32 m, const ulonglong2 *tw,
                                                 u64 p, u64 two_p, std::integer_sequence<int, Q...>)
{
    (fwd_stage<Sh, Rd, Q>(x, tid, m, tw, p, two_p), ...);
}

template <class Sh, class Rd>
__device__ __forceinline__ void fwd_round_compute(u64 (&x)[16], u32 tid, u32 m, const ulonglong2 *tw,
                                                  u64 p, u64 two_p)
{
    fwd_round_stages<Sh, Rd>(x, tid, m, tw, p, two_p, std::make_integer_sequence<int, Rd::R>{});
}

template <class Sh, class Rd>
__device__ __forceinline__ void round_load_smem(u64 (&x)[16], const u64 *s, u32 tid)
{
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++)
#pragma unroll
        for (int u = 0; u < (1 << Rd::R); u++) x[i * (1 << Rd::R) + u] = s[swz(round_pos<Rd>(tid, i, u))];
}

template <class Sh, class Rd>
__device__ __forceinline__ void round_store_smem(const u64 (&x)[16], u64 *s, u32 tid)
{
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++)
#pragma unroll
        for (int u = 0; u < (1 << Rd::R); u++) s[swz(round_pos<Rd>(tid, i, u))] = x[i * (1 << Rd::R) + u];
}

template <class Sh, int RI>
struct RoundOf {
    using type = Round<(RI < Sh::NROUND - 1) ? 4 : Sh::LAST_R, 4 * RI, Sh::LOG_B>;
};

// Cross-CTA stages of the forward transform: load columns, radix-C network,
// scatter into the owning CTAs' shared memory, cluster barrier.
template <class Sh, class Load>
__device__ __forceinline__ void fwd_cross(u64 *s, u32 tid, u32 m, const ulonglong2 *tw, u64 p, u64 two_p,
                                          Load &load)
{
    constexpr u32 C = Sh::C;
    constexpr int COLS = 16 / (int)C;
    ulonglong2 wt[C];
#pragma unroll
    for (u32 i = 1; i < C; i++) wt[i] = ld_tw(tw, i);
    const u32 s_base = smem_u32(s);
#pragma unroll
    for (int c = 0; c < COLS; c++) {
        u32 j = m * (Sh::B / C) + (u32)c * Sh::T + tid;
        u64 v[C];
#pragma unroll
        for (u32 t = 0; t < C; t++) v[t] = load(t * Sh::B + j);
#pragma unroll
        for (int S = 0; S < Sh::LOG_C; S++) {
            const u32 half = C >> (S + 1);
#pragma unroll
            for (u32 t = 0; t < C; t++) {
                if (t & half) continue;
                u32 idx = (1u << S) + (t >> (Sh::LOG_C - S));
                ct_butterfly(v[t], v[t + half], wt[idx].x, wt[idx].y, p, two_p);
            }
        }
        u32 a = s_base + swz(j) * 8u;
#pragma unroll
        for (u32 t = 0; t < C; t++) st_cluster(map_to_rank(a, t), v[t]);
    }
    cluster_sync_all();
}

// Forward negacyclic NTT of one limb. load(P) gives input position P in
// [0, N) (values below 4p); store(P, v) receives the canonical output at
// bit-reversed evaluation index P. After the call the values also remain in
// x[] in the last round's order (round_pos of the last round), canonical.
template <class Sh, class Load, class Store>
__device__ __forceinline__ void ntt_fwd_block(u64 *s, u32 m, const ulonglong2 *tw, u64 p, u64 two_p,
                                              Load load, Store store, u64 (&x)[16])
{
    const u32 tid = threadIdx.x;
    using R0 = typename RoundOf<Sh, 0>::type;
    using R1 = typename RoundOf<Sh, (Sh::NROUND > 1 ? 1 : 0)>::type;
    using R2 = typename RoundOf<Sh, (Sh::NROUND > 2 ? 2 : 0)>::type;
    using R3 = typename RoundOf<Sh, (Sh::NROUND > 3 ? 3 : 0)>::type;

    if constexpr (Sh::LOG_C > 0) {
        fwd_cross<Sh>(s, tid, m, tw, p, two_p, load);
        round_load_smem<Sh, R0>(x, s, tid);
    } else {
#pragma unroll
        for (int i = 0; i < R0::SUB; i++)
#pragma unroll
            for (int u = 0; u < (1 << R0::R); u++) x[i * (1 << R0::R) + u] = load(round_pos<R0>(tid, i, u));
    }
    fwd_round_compute<Sh, R0>(x, tid, m, tw, p, two_p);
    using RL = typename RoundOf<Sh, Sh::NROUND - 1>::type;
    if constexpr (Sh::NROUND > 1) {
        round_store_smem<Sh, R0>(x, s, tid);
        __syncthreads();
        round_load_smem<Sh, R1>(x, s, tid);
        fwd_round_compute<Sh, R1>(x, tid, m, tw, p, two_p);
    }
    if constexpr (Sh::NROUND > 2) {
        round_store_smem<Sh, R1>(x, s, tid);
        __syncthreads();
        round_load_smem<Sh, R2>(x, s, tid);
        fwd_round_compute<Sh, R2>(x, tid, m, tw, p, two_p);
    }
    if constexpr (Sh::NROUND > 3) {
        round_store_smem<Sh, R2>(x, s, tid);
        __syncthreads();
        round_load_smem<Sh, R3>(x, s, tid);
        fwd_round_compute<Sh, R3>(x, tid, m, tw, p, two_p);
    }
    static_assert(Sh::NROUND <= 4, "at most four local rounds");
#pragma unroll
    for (int i = 0; i < RL::SUB; i++)
#pragma unroll
        for (int u = 0; u < (1 << RL::R); u++) {
            u64 v = reduce_once(reduce_once(x[i * (1 << RL::R) + u], two_p), p);
            x[i * (1 << RL::R) + u] = v;
            store(m * Sh::B + round_pos<RL>(tid, i, u), v);
        }
}

// ---------------------------------------------------------------- inverse

// The final inverse stage (S = 0, one group, gap N/2) with N^-1 folded in:
// (x, y) -> ((x + y) N^-1, (x - y) psi^-brv(1) N^-1), canonical outputs.
__device__ __forceinline__ void gs_last(u64 &x, u64 &y, const PrimeConst &pc)
{
    u64 X = mul_shoup(x + y, pc.ninv, pc.ninv_sh, pc.p);
    u64 Y = mul_shoup(x - y + pc.two_p, pc.w1ninv, pc.w1ninv_sh, pc.p);
    x = X;
    y = Y;
}

template <class Sh, class Rd, int q>
__device__ __forceinline__ void inv_stage(u64 (&x)[16], u32 tid, u32 m, const ulonglong2 *tw,
                                          const PrimeConst &pc)
{
    constexpr int S = Sh::LOG_C + Rd::S0 + q;
    constexpr int half = 1 << (Rd::R - 1 - q);
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++) {
        const u32 G = round_group_base<Sh, Rd>(tid, i, m);
#pragma unroll
        for (int grp = 0; grp < (1 << q); grp++) {
            if constexpr (S == 0) {
#pragma unroll
                for (int v = 0; v < half; v++) {
                    const int u = grp * 2 * half + v;
                    gs_last(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], pc);
                }
            } else {
                const ulonglong2 w = ld_tw(tw, (1u << S) + (G << q) + (u32)grp);
#pragma unroll
                for (int v = 0; v < half; v++) {
                    const int u = grp * 2 * half + v;
                    gs_butterfly(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], w.x, w.y, pc.p,
                                 pc.two_p);
                }
            }
        }
    }
}

// Stages of an inverse round run in decreasing order (increasing gap).
template <class Sh, class Rd, int... Q>
__device__ __forceinline__ void inv_round_stages(u64 (&x)[16], u32 tid, u32 m, const ulonglong2 *tw,
                                                 const PrimeConst &pc, std::integer_sequence<int, Q...>)
{
    (inv_stage<Sh, Rd, Rd::R - 1 - Q>(x, tid, m, tw, pc), ...);
}

template <class Sh, class Rd>
__device__ __forceinline__ void inv_round_compute(u64 (&x)[16], u32 tid, u32 m, const ulonglong2 *tw,
                                                  const PrimeConst &pc)
{
    inv_round_stages<Sh, Rd>(x, tid, m, tw, pc, std::make_integer_sequence<int, Rd::R>{});
}

// Inverse negacyclic NTT (with N^-1) of one limb. If the caller already
// holds the block's values in x[] in the forward transform's last-round
// order, pass have_x = true and load is not called; otherwise load(P) gives
// the NTT-domain value at position P (below 2p). store(P, v) receives the
// canonical coefficient P.
template <class Sh, bool HAVE_X, class Load, class Store>
__device__ __forceinline__ void ntt_inv_block(u64 *s, u32 m, const ulonglong2 *tw, const PrimeConst &pc,
                                              Load load, Store store, u64 (&x)[16])
{
    const u32 tid = threadIdx.x;
    constexpr int NR = Sh::NROUND;
    using RL = typename RoundOf<Sh, NR - 1>::type;
    using RL1 = typename RoundOf<Sh, (NR >= 2 ? NR - 2 : 0)>::type;
    using RL2 = typename RoundOf<Sh, (NR >= 3 ? NR - 3 : 0)>::type;
    using RL3 = typename RoundOf<Sh, (NR >= 4 ? NR - 4 : 0)>::type;
    static_assert(NR >= 2 && NR <= 4, "two to four local rounds");

    if constexpr (!HAVE_X) {
#pragma unroll
        for (int i = 0; i < RL::SUB; i++)
#pragma unroll
            for (int u = 0; u < (1 << RL::R); u++)
                x[i * (1 << RL::R) + u] = load(m * Sh::B + round_pos<RL>(tid, i, u));
    }
    inv_round_compute<Sh, RL>(x, tid, m, tw, pc);
    round_store_smem<Sh, RL>(x, s, tid);
    __syncthreads();
    round_load_smem<Sh, RL1>(x, s, tid);
    inv_round_compute<Sh, RL1>(x, tid, m, tw, pc);
    if constexpr (NR > 2) {
        round_store_smem<Sh, RL1>(x, s, tid);
        __syncthreads();
        round_load_smem<Sh, RL2>(x, s, tid);
        inv_round_compute<Sh, RL2>(x, tid, m, tw, pc);
    }
    if constexpr (NR > 3) {
        round_store_smem<Sh, RL2>(x, s, tid);
        __syncthreads();
        round_load_smem<Sh, RL3>(x, s, tid);
        inv_round_compute<Sh, RL3>(x, tid, m, tw, pc);
    }
    using R0 = typename RoundOf<Sh, 0>::type;
    if constexpr (Sh::LOG_C == 0) {
        // round 0 ended with the final stage: values are canonical
#pragma unroll
        for (int i = 0; i < R0::SUB; i++)
#pragma unroll
            for (int u = 0; u < (1 << R0::R); u++) store(round_pos<R0>(tid, i, u), x[i * (1 << R0::R) + u]);
    } else {
        round_store_smem<Sh, R0>(x, s, tid);
        cluster_sync_all();
        constexpr u32 C = Sh::C;
        constexpr int COLS = 16 / (int)C;
        ulonglong2 wt[C];
#pragma unroll
        for (u32 i = 2; i < C; i++) wt[i] = ld_tw(tw, i);
        const u32 s_base = smem_u32(s);
#pragma unroll
        for (int c = 0; c < COLS; c++) {
            u32 j = m * (Sh::B / C) + (u32)c * Sh::T + tid;
            u32 a = s_base + swz(j) * 8u;
            u64 v[C];
#pragma unroll
            for (u32 t = 0; t < C; t++) v[t] = ld_cluster(map_to_rank(a, t));
#pragma unroll
            for (int SS = 0; SS < Sh::LOG_C; SS++) {
                const int S = Sh::LOG_C - 1 - SS;
                const u32 half = C >> (S + 1);
#pragma unroll
                for (u32 t = 0; t < C; t++) {
                    if (t & half) continue;
                    if (S == 0) {
                        gs_last(v[t], v[t + half], pc);
                    } else {
                        u32 idx = (1u << S) + (t >> (Sh::LOG_C - S));
                        gs_butterfly(v[t], v[t + half], wt[idx].x, wt[idx].y, pc.p, pc.two_p);
                    }
                }
            }
#pragma unroll
            for (u32 t = 0; t < C; t++) store(t * Sh::B + j, v[t]);
        }
        cluster_sync_all();  // peers may still read this CTA's shared memory
    }
}

}  // namespace he
