// ntt_core.cuh -- block-level negacyclic NTT building blocks for sm_103a.
//
// One limb of N = B * C words is transformed by C CTAs of a thread-block
// cluster; CTA m owns the contiguous block [m B, (m + 1) B) of positions in
// shared memory (B = 2^LOG_B words, E = 2^LOG_E words per thread).
//
// Forward transform (Sec. II-B with the psi twist folded into bit-reversed
// twiddles; Cooley-Tukey stages with Harvey's lazy butterfly, Algorithm 1,
// here on the range [0, 8p + 2^32), see modarith.cuh):
//   stage S (0 .. log N - 1) has 2^S groups of 2 N / 2^S positions; group g
//   uses W = psi^brv(2^S + g) and pairs positions j and j + N / 2^(S+1).
//   * The first log C stages pair positions in different CTAs. Each thread
//     loads whole columns {t B + j : t < C} from global memory, runs the
//     radix-C network in registers and hands element t to CTA t through
//     distributed shared memory: scattered with st.shared::cluster, or (16
//     words per thread) kept locally for CTA t to read with
//     ld.shared::cluster. This is the paper's "global memory" stage group,
//     done without a second pass over HBM.
//   * The remaining log B stages stay inside one CTA: rounds of up to LOG_E
//     stages (radix E) in registers, exchanging through shared memory
//     between rounds (the paper's SLM rounds, Sec. III-B; its best radix was
//     8, here radix 8 and radix 16 are both built and the autotuner picks).
//   * The last round reduces to [0, p) (the paper's last-round
//     offsetting, fused) and hands each canonical value to the caller's store
//     functor.
// Inverse transform: the mirror image with Gentleman-Sande butterflies on
// [0, 4p); local rounds first, cross-CTA stages last, N^-1 folded into the
// final stage.
//
// Shared-memory layout: element l of the block sits at word l ^ f(l >> 4)
// for a per-radix f (a permutation inside each 16-word row) that keeps every
// access pattern below free of bank conflicts: each half warp touches 16
// distinct 8-byte bank pairs.
#pragma once
#include <stdint.h>

#include <utility>

#include "modarith.cuh"

namespace he {

template <int LOG_E>
__device__ __forceinline__ u32 swz(u32 l);

template <>
__device__ __forceinline__ u32 swz<4>(u32 l)
{
    return l ^ ((l >> 4) & 15u);
}

template <>
__device__ __forceinline__ u32 swz<3>(u32 l)
{
    const u32 r = l >> 4;
    return l ^ (((r ^ ((r >> 1) << 2)) * 9u) & 15u);
}

// threadIdx.x, with the launch's block size made known to the compiler: the
// transforms always run T = B / E threads a CTA, so round 0's group index
// (tid >> log2 T) folds to 0 and its twiddle addresses become CTA-uniform.
// Used by the inverse transform, where it measured 1.5 % faster (the forward
// transform measured 2 % slower with it).
template <u32 T>
__device__ __forceinline__ u32 thread_index()
{
    const u32 t = threadIdx.x;
    __builtin_assume(t < T);
    return t;
}

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

// Cluster barrier for write-after-read only: every CTA has finished reading
// shared memory that a peer is about to overwrite (or release by exiting).
// Those reads have returned their values before the arrive is issued, so the
// arrive needs no release ordering (and no memory fence before it); waits on
// it still acquire. The callers make sure of that: ntt_barrier between two
// transforms follows the first one's closing barrier (which already waited
// for its remote reads); the transforms' own barriers after remote reads
// tie the arrive to the words read (cluster_sync_war_fold / _after).
__device__ __forceinline__ void cluster_sync_war()
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// cluster_sync_war for a thread whose last reads of peers' shared memory
// produced x[] (remote loads, then register arithmetic): the arrive takes
// a fold of every word as an operand, so the compiler cannot sink the
// arithmetic past it and, a warp issuing in order, the arrive cannot issue
// before the remote loads have returned.
__device__ __forceinline__ void cluster_sync_war_fold(u64 f)
{
    asm volatile("barrier.cluster.arrive.relaxed.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::"l"(f) : "memory");
}

template <int E>
__device__ __forceinline__ void cluster_sync_war_after(const u64 (&x)[E])
{
    u64 f = x[0];
#pragma unroll
    for (int e = 1; e < E; e++) f |= x[e];
    cluster_sync_war_fold(f);
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

// Positions and twiddle indices are signed ints (all below 2^17): a signed
// sum cannot wrap, so the compiler may split base + constant and fold the
// constant into the load's immediate offset, where a u32 sum would need its
// own 64-bit address computation per access.
__device__ __forceinline__ ulonglong2 ld_tw(const ulonglong2 *tw, int idx) { return __ldg(tw + idx); }

// Two consecutive twiddle pairs (idx even, so 32-byte aligned: tables start
// 256-byte aligned and hold N pairs per prime) in one 256-bit load. Half the
// load instructions of two 128-bit loads, which measured clearly faster:
// the per-stage twiddle loads, not their latency, are what the transform's
// local rounds pay for beyond the butterflies.
__device__ __forceinline__ void ld_tw2(const ulonglong2 *tw, int idx, ulonglong2 &a, ulonglong2 &b)
{
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(a.x), "=l"(a.y), "=l"(b.x), "=l"(b.y)
        : "l"(tw + idx));
}

// Position of the inverse twiddle psi^-brv(2^S + G) (stage S, group G <
// 2^S) in its table of N pairs. Stages S < log N - 4 keep the natural order
// 2^S + G. In each of the last four stages (Q = S - (log N - 4) = 0..3,
// 2^(log N - 4) runs of 2^Q groups) group G = t 2^Q + r goes to
//   2^S + (r >> 1) 2^(log N - 3) + 2 t + (r & 1):
// the run-major order turned run-minor, keeping pairs (r, r + 1) with r even
// adjacent. The inverse transform's first round hands thread t of the
// transform (across the cluster) the groups t 2^Q .. t 2^Q + 2^Q - 1 of
// stage log N - 4 + Q, so its 256-bit loads of two pairs become lane-
// consecutive (1 KB per warp instead of 32 separate lines; measured 2.3 %
// off the inverse at N = 2^15). The forward table keeps the natural order
// (the same layout measured no faster there). For Q >= 1 the position of
// an even G is even, so the pair G, G + 1 stays one aligned 32-byte load.
__host__ __device__ __forceinline__ int inv_tw_pos(int log_n, int S, int G)
{
    const int Q = S - (log_n - 4);
    if (Q <= 0) return (1 << S) + G;
    const int t = G >> Q, r = G & ((1 << Q) - 1);
    return (1 << S) + ((r >> 1) << (log_n - 3)) + 2 * t + (r & 1);
}

// 256-bit global accesses (sm_100 and later): four consecutive words at a
// 32-byte aligned address. A thread's run of words in the forward
// transform's last round and the inverse transform's first round starts at
// m B + tid E, so its quarters (e = 0 mod 4) are 32-byte aligned in every
// buffer that is, and the library requires 32-byte aligned device buffers.
// Each lane's run lies in its own 128-byte line, so one 256-bit access
// costs the L1 what one 128-bit access did: half the requests for the same
// words (measured 4-5 % off both transform directions at N = 2^15).
// _cs: streaming (data read or written once per launch); _nc: read-only
// path (data that no thread of the launch writes).
__device__ __forceinline__ void ld4_cs(const u64 *p, u64 &a, u64 &b, u64 &c, u64 &d)
{
    asm("ld.global.cs.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

__device__ __forceinline__ void ld4_nc(const u64 *p, u64 &a, u64 &b, u64 &c, u64 &d)
{
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

// A plain load: the memory clobber keeps it ordered after this thread's
// earlier stores (the caller may read a buffer it has just written).
__device__ __forceinline__ void ld4(const u64 *p, u64 &a, u64 &b, u64 &c, u64 &d)
{
    asm volatile("ld.global.v4.u64 {%0, %1, %2, %3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p) : "memory");
}

__device__ __forceinline__ void st4_cs(u64 *p, u64 a, u64 b, u64 c, u64 d)
{
    asm volatile("st.global.cs.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}

__device__ __forceinline__ void st4(u64 *p, u64 a, u64 b, u64 c, u64 d)
{
    asm volatile("st.global.v4.u64 [%0], {%1, %2, %3, %4};" ::"l"(p), "l"(a), "l"(b), "l"(c), "l"(d) : "memory");
}

// OCC_: CTAs per SM the transform kernels are compiled for (their register
// budget); 0 = the shape's default below.
template <int LOG_B_, int LOG_C_, int LOG_E_ = 4, int OCC_ = 0>
struct NttShape {
    static constexpr int LOG_B = LOG_B_;
    static constexpr int LOG_C = LOG_C_;
    static constexpr int LOG_E = LOG_E_;
    static constexpr int LOG_N = LOG_B + LOG_C;
    static constexpr u32 B = 1u << LOG_B;
    static constexpr u32 C = 1u << LOG_C;
    static constexpr u32 N = 1u << LOG_N;
    static constexpr int E = 1 << LOG_E;          // words per thread
    static constexpr u32 T = B / E;               // threads per CTA
    static constexpr int NROUND = (LOG_B + LOG_E - 1) / LOG_E;
    static constexpr int LAST_R = LOG_B - LOG_E * (NROUND - 1);
    static constexpr u32 SMEM_BYTES = B * 8;
    // Exchange of the forward transform's cross-CTA stages: push (each CTA
    // stores its results into the owners' shared memory, one cluster
    // barrier) or pull (each CTA keeps them, one cluster barrier, the owners
    // read them remotely, and a second barrier before the block is reused,
    // after the first register round). Pull measured 3 % faster with 16
    // words per thread and 11 % slower with 8 (N = 2^15).
    static constexpr bool FWD_PULL = LOG_E == 4;
    // CTAs per SM to aim for, from a register budget per thread: occupancy
    // pays for the transform (measured: radix-8 at 42 registers, three 512-
    // thread CTAs per SM, beats 64 registers by 8-9%; radix-16 at 64
    // registers, four 256-thread CTAs, beats 128 by 7-18%), even with the
    // few spills these budgets cost
    static constexpr int REGS = LOG_E == 4 ? 64 : 42;
    static constexpr int MIN_CTAS =
        OCC_ > 0 ? OCC_ : ((65536 / (int)(T * REGS)) > 0 ? 65536 / (int)(T * REGS) : 1);
    // evaluation kernels carry more state per thread: 128 registers
    static constexpr int EVAL_MIN_CTAS = (65536 / (int)(T * 128)) > 0 ? 65536 / (int)(T * 128) : 1;
    // the fused product (three transforms, a second shared-memory block):
    // 80 registers with 16 words per thread (three CTAs per SM, which its
    // shared memory allows anyway), 64 with 8
    static constexpr int NEGA_REGS = LOG_E == 4 ? 80 : 64;
    static constexpr int NEGA_MIN_CTAS = (65536 / (int)(T * NEGA_REGS)) > 0 ? 65536 / (int)(T * NEGA_REGS) : 1;
    static_assert(LOG_C <= 4, "clusters of at most 16 CTAs (more than 8: the non-portable size)");
    static_assert(LOG_C <= LOG_E, "a thread holds whole columns of the cross stages");
    static_assert(LOG_E == 3 || LOG_E == 4, "radix 8 or 16 rounds");
    static_assert(T >= 32 && T <= 1024, "one to 32 warps per CTA");
};

// Round RI of the local stages: R stages starting at local stage S0; each
// thread holds SUB subgroups of 2^R words spaced TL apart.
template <class Sh, int RI>
struct RoundOf {
    static constexpr int R = (RI < Sh::NROUND - 1) ? Sh::LOG_E : Sh::LAST_R;
    static constexpr int S0 = Sh::LOG_E * RI;
    static constexpr int SUB = Sh::E >> R;
    static constexpr int LOG_TL = Sh::LOG_B - S0 - R;
    static constexpr u32 TL = 1u << LOG_TL;
};

// Threads that exchange words between round RI and round RI + 1 (in either
// direction): a group of round RI, i.e. positions g 2^(LOG_TL + R) + k +
// u TL for all k < TL and u, is held by TL / SUB consecutive threads in round
// RI, and every group of round RI + 1 lies inside one group of round RI. So
// the exchange needs no more than those threads to meet: the whole CTA, a
// named barrier of 64 or 128 threads, or the warp. (Each thread only ever
// overwrites the shared-memory words it read itself in the previous
// exchange, so there is no write-after-read hazard across groups.)
template <class Sh, int RI>
struct RoundLink {
    using Rd = RoundOf<Sh, RI>;
    static constexpr u32 THREADS = Rd::TL / Rd::SUB;
    static_assert(THREADS >= 1 && (Sh::T % (THREADS < 32 ? 32 : THREADS)) == 0, "groups tile the CTA");
    static_assert(THREADS <= 32 || THREADS >= Sh::T || Sh::T / THREADS <= 15, "named barrier ids 1..15");
};

template <class Sh, int RI>
__device__ __forceinline__ void round_link_sync(u32 tid)
{
    constexpr u32 G = RoundLink<Sh, RI>::THREADS;
    if constexpr (G >= Sh::T) {
        __syncthreads();
    } else if constexpr (G <= 32) {
        __syncwarp();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1u + tid / G), "n"(G) : "memory");
    }
}

// Block-local position of element u of subgroup i of this thread in a round.
template <class Rd>
__device__ __forceinline__ int round_pos(u32 tid, int i, int u)
{
    const int sg = (int)tid * Rd::SUB + i;
    const int k = sg & ((int)Rd::TL - 1);
    const int g = sg >> Rd::LOG_TL;
    return g * (1 << (Rd::LOG_TL + Rd::R)) + k + u * (int)Rd::TL;
}

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

// Barrier between two consecutive block transforms in one CTA: the next
// transform's first writes to shared memory (remote ones for a cluster) must
// not overtake reads of the previous transform.
template <class Sh>
__device__ __forceinline__ void ntt_barrier()
{
    if constexpr (Sh::LOG_C > 0)
        cluster_sync_war();
    else
        __syncthreads();
}

// Shared-memory word index of element u of subgroup i in a round. Both
// swizzles are linear over GF(2) and the subgroup base and u * TL occupy
// disjoint bits (base = g << (LOG_TL + R) | k with k < TL), so
// swz(base + u TL) = swz(base) ^ swz(u << LOG_TL): one per-thread term and
// a compile-time constant per element.
template <class Sh, class Rd>
__device__ __forceinline__ u32 round_base_swz(u32 tid, int i)
{
    return swz<Sh::LOG_E>(round_pos<Rd>(tid, i, 0));
}

template <class Sh, class Rd>
__device__ __forceinline__ void round_load_smem(u64 (&x)[Sh::E], const u64 *s, u32 tid)
{
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++) {
        const u32 pb = round_base_swz<Sh, Rd>(tid, i);
#pragma unroll
        for (int u = 0; u < (1 << Rd::R); u++)
            x[i * (1 << Rd::R) + u] = s[pb ^ swz<Sh::LOG_E>((u32)u << Rd::LOG_TL)];
    }
}

template <class Sh, class Rd>
__device__ __forceinline__ void round_store_smem(const u64 (&x)[Sh::E], u64 *s, u32 tid)
{
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++) {
        const u32 pb = round_base_swz<Sh, Rd>(tid, i);
#pragma unroll
        for (int u = 0; u < (1 << Rd::R); u++)
            s[pb ^ swz<Sh::LOG_E>((u32)u << Rd::LOG_TL)] = x[i * (1 << Rd::R) + u];
    }
}

// ---------------------------------------------------------------- forward

// CANON_OUT: this is the transform's last stage and its outputs must be
// canonical (ct_butterfly_canon); otherwise the lazy butterfly.
template <class Sh, class Rd, int q, bool CANON_OUT>
__device__ __forceinline__ void fwd_stage(u64 (&x)[Sh::E], u32 tid, u32 m, const ulonglong2 *tw,
                                          const PrimeConst &pc)
{
    constexpr int S = Sh::LOG_C + Rd::S0 + q;     // global stage
    constexpr int half = 1 << (Rd::R - 1 - q);
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++) {
        const u32 G = round_group_base<Sh, Rd>(tid, i, m);
        ulonglong2 ws[1 << q];
        if constexpr (q == 0) {
            ws[0] = ld_tw(tw, (1 << S) + (int)G);
        } else {
#pragma unroll
            for (int grp = 0; grp < (1 << q); grp += 2) ld_tw2(tw, (1 << S) + (int)G * (1 << q) + grp, ws[grp], ws[grp + 1]);
        }
#pragma unroll
        for (int grp = 0; grp < (1 << q); grp++) {
            const ulonglong2 w = ws[grp];
#pragma unroll
            for (int v = 0; v < half; v++) {
                const int u = grp * 2 * half + v;
                if constexpr (CANON_OUT)
                    ct_butterfly_canon(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], w.x, w.y, pc);
                else
                    ct_butterfly(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], w.x, w.y, pc);
            }
        }
    }
}

template <class Sh, class Rd, bool CANON_LAST, int... Q>
__device__ __forceinline__ void fwd_round_stages(u64 (&x)[Sh::E], u32 tid, u32 m, const ulonglong2 *tw,
                                                 const PrimeConst &pc, std::integer_sequence<int, Q...>)
{
    (fwd_stage<Sh, Rd, Q, CANON_LAST && Q == Rd::R - 1>(x, tid, m, tw, pc), ...);
}

template <class Sh, int RI, bool CANON>
__device__ __forceinline__ void fwd_round(u64 (&x)[Sh::E], u64 *s, u32 tid, u32 m, const ulonglong2 *tw,
                                          const PrimeConst &pc)
{
    using Rd = RoundOf<Sh, RI>;
    if constexpr (RI > 0) {
        // pull form: the peers have pulled their words out of this block
        if constexpr (RI == 1 && Sh::LOG_C > 0 && Sh::FWD_PULL) cluster_sync_war_after(x);
        round_store_smem<Sh, RoundOf<Sh, RI - 1>>(x, s, tid);
        round_link_sync<Sh, RI - 1>(tid);
        round_load_smem<Sh, Rd>(x, s, tid);
    }
    fwd_round_stages<Sh, Rd, CANON && RI == Sh::NROUND - 1>(x, tid, m, tw, pc,
                                                            std::make_integer_sequence<int, Rd::R>{});
}

template <class Sh, bool CANON, int... RI>
__device__ __forceinline__ void fwd_rounds(u64 (&x)[Sh::E], u64 *s, u32 tid, u32 m, const ulonglong2 *tw,
                                           const PrimeConst &pc, std::integer_sequence<int, RI...>)
{
    (fwd_round<Sh, RI, CANON>(x, s, tid, m, tw, pc), ...);
}

// Cross-CTA stages of the forward transform: load columns, radix-C network,
// then either scatter into the owning CTAs' shared memory (ranks rbase ..
// rbase + C - 1 of the cluster) or keep the results for the owners to pull
// (Sh::FWD_PULL), cluster barrier.
template <class Sh, class Load>
__device__ __forceinline__ void fwd_cross(u64 *s, u32 tid, u32 m, u32 rbase, const ulonglong2 *tw,
                                          const PrimeConst &pc, Load &load)
{
    constexpr u32 C = Sh::C;
    constexpr int COLS = Sh::E / (int)C;
    const u32 s_base = smem_u32(s);
#pragma unroll
    for (int c = 0; c < COLS; c++) {
        const int j = (int)(m * (Sh::B / C)) + c * (int)Sh::T + (int)tid;
        u64 v[C];
#pragma unroll
        for (u32 t = 0; t < C; t++) v[t] = load((int)t * (int)Sh::B + j);
#pragma unroll
        for (int S = 0; S < Sh::LOG_C; S++) {
            const u32 half = C >> (S + 1);
            ulonglong2 ws[C / 2];   // this stage's twiddles only: fewer live registers
#pragma unroll
            for (int g = 0; g < (1 << S); g++) ws[g] = ld_tw(tw, (1 << S) + g);
#pragma unroll
            for (u32 t = 0; t < C; t++) {
                if (t & half) continue;
                const ulonglong2 w = ws[t >> (Sh::LOG_C - S)];
                ct_butterfly(v[t], v[t + half], w.x, w.y, pc);
            }
        }
        if constexpr (Sh::FWD_PULL) {
            // kept in this CTA's block, word t of column offset o at
            // t B / C + o, for the owner of the column's words to pull
            const int o = c * (int)Sh::T + (int)tid;
#pragma unroll
            for (u32 t = 0; t < C; t++) s[((int)t << (Sh::LOG_B - Sh::LOG_C)) + o] = v[t];
        } else {
            const u32 a = s_base + swz<Sh::LOG_E>((u32)j) * 8u;
#pragma unroll
            for (u32 t = 0; t < C; t++) st_cluster(map_to_rank(a, rbase + t), v[t]);
        }
    }
    cluster_sync_all();
}

// Forward negacyclic NTT of one limb. m is this CTA's block (rank within its
// group of C CTAs, which sit at cluster ranks rbase .. rbase + C - 1).
// load(P) gives input position P in [0, N) (values below 8p); store(P, v)
// receives the canonical output at bit-reversed evaluation index P. After
// the call the canonical values also remain in x[] in the last round's order
// (see last_pos). With CANON = false the final reduction is skipped: x[] and
// store receive values in [0, 8p + 2^32), below 12p for p >= 2^30, for
// callers that feed them straight into a Shoup product (any 64-bit input).
template <class Sh, bool CANON = true, class Load, class Store>
__device__ __forceinline__ void ntt_fwd_block(u64 *s, u32 m, u32 rbase, const ulonglong2 *tw,
                                              const PrimeConst &pc, Load load, Store store, u64 (&x)[Sh::E])
{
    const u32 tid = threadIdx.x;
    using R0 = RoundOf<Sh, 0>;
    if constexpr (Sh::LOG_C > 0) {
        fwd_cross<Sh>(s, tid, m, rbase, tw, pc, load);
        if constexpr (Sh::FWD_PULL) {
            constexpr int LOG_W = Sh::LOG_B - Sh::LOG_C;
            const u32 s_base = smem_u32(s);
#pragma unroll
            for (int i = 0; i < R0::SUB; i++)
#pragma unroll
                for (int u = 0; u < (1 << R0::R); u++) {
                    const int P = round_pos<R0>(tid, i, u);
                    const u32 slot = (m << LOG_W) + ((u32)P & ((1u << LOG_W) - 1));
                    x[i * (1 << R0::R) + u] = ld_cluster(map_to_rank(s_base + slot * 8u, rbase + ((u32)P >> LOG_W)));
                }
            if constexpr (Sh::NROUND == 1) cluster_sync_war_after(x);   // peers pulled from this block
        } else {
            round_load_smem<Sh, R0>(x, s, tid);
        }
    } else {
#pragma unroll
        for (int i = 0; i < R0::SUB; i++)
#pragma unroll
            for (int u = 0; u < (1 << R0::R); u++) x[i * (1 << R0::R) + u] = load(round_pos<R0>(tid, i, u));
    }
    fwd_rounds<Sh, CANON>(x, s, tid, m, tw, pc, std::make_integer_sequence<int, Sh::NROUND>{});
    using RL = RoundOf<Sh, Sh::NROUND - 1>;
#pragma unroll
    for (int i = 0; i < RL::SUB; i++)
#pragma unroll
        for (int u = 0; u < (1 << RL::R); u++)
            store((int)(m * Sh::B) + round_pos<RL>(tid, i, u), x[i * (1 << RL::R) + u]);
}

// Position (within the limb) of element e of x[] after ntt_fwd_block, and of
// the input element e expected by ntt_inv_block with HAVE_X.
template <class Sh>
__device__ __forceinline__ int last_pos(u32 m, u32 tid, int e)
{
    using RL = RoundOf<Sh, Sh::NROUND - 1>;
    return (int)(m * Sh::B) + round_pos<RL>(tid, e >> RL::R, e & ((1 << RL::R) - 1));
}

// ---------------------------------------------------------------- inverse

// The final inverse stage (S = 0, one group, gap N/2) with N^-1 folded in:
// (x, y) -> ((x + y) N^-1, (x - y) psi^-brv(1) N^-1), canonical outputs
// (inputs in [0, 4p); the lazy products land in [0, 4p) and reduce twice).
__device__ __forceinline__ void gs_last(u64 &x, u64 &y, const PrimeConst &pc)
{
    const u64 X = mul_shoup_lazy4(x + y, pc.ninv, pc.ninv_sh, pc.neg_p);
    const u64 Y = mul_shoup_lazy4(x - y + pc.four_p, pc.w1ninv, pc.w1ninv_sh, pc.neg_p);
    x = reduce_once(reduce_once(X, pc.two_p), pc.p);
    y = reduce_once(reduce_once(Y, pc.two_p), pc.p);
}

template <class Sh, class Rd, int q>
__device__ __forceinline__ void inv_stage(u64 (&x)[Sh::E], u32 tid, u32 m, const ulonglong2 *tw,
                                          const PrimeConst &pc)
{
    constexpr int S = Sh::LOG_C + Rd::S0 + q;
    constexpr int half = 1 << (Rd::R - 1 - q);
#pragma unroll
    for (int i = 0; i < Rd::SUB; i++) {
        const u32 G = round_group_base<Sh, Rd>(tid, i, m);
        ulonglong2 ws[1 << q];
        if constexpr (S > 0) {
            if constexpr (q == 0) {
                ws[0] = ld_tw(tw, inv_tw_pos(Sh::LOG_N, S, (int)G));
            } else {
#pragma unroll
                for (int grp = 0; grp < (1 << q); grp += 2)
                    ld_tw2(tw, inv_tw_pos(Sh::LOG_N, S, (int)G * (1 << q) + grp), ws[grp], ws[grp + 1]);
            }
        }
#pragma unroll
        for (int grp = 0; grp < (1 << q); grp++) {
            if constexpr (S == 0) {
#pragma unroll
                for (int v = 0; v < half; v++) {
                    const int u = grp * 2 * half + v;
                    gs_last(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], pc);
                }
            } else {
                const ulonglong2 w = ws[grp];
#pragma unroll
                for (int v = 0; v < half; v++) {
                    const int u = grp * 2 * half + v;
                    gs_butterfly(x[i * (1 << Rd::R) + u], x[i * (1 << Rd::R) + u + half], w.x, w.y, pc);
                }
            }
        }
    }
}

// Stages of an inverse round run in decreasing order (increasing gap).
template <class Sh, class Rd, int... Q>
__device__ __forceinline__ void inv_round_stages(u64 (&x)[Sh::E], u32 tid, u32 m, const ulonglong2 *tw,
                                                 const PrimeConst &pc, std::integer_sequence<int, Q...>)
{
    (inv_stage<Sh, Rd, Rd::R - 1 - Q>(x, tid, m, tw, pc), ...);
}

// Inverse rounds run from the last local round down to round 0.
template <class Sh, int RI>
__device__ __forceinline__ void inv_round(u64 (&x)[Sh::E], u64 *s, u32 tid, u32 m, const ulonglong2 *tw,
                                          const PrimeConst &pc)
{
    using Rd = RoundOf<Sh, RI>;
    if constexpr (RI < Sh::NROUND - 1) {
        round_store_smem<Sh, RoundOf<Sh, RI + 1>>(x, s, tid);
        round_link_sync<Sh, RI>(tid);
        round_load_smem<Sh, Rd>(x, s, tid);
    }
    inv_round_stages<Sh, Rd>(x, tid, m, tw, pc, std::make_integer_sequence<int, Rd::R>{});
}

template <class Sh, int... Q>
__device__ __forceinline__ void inv_rounds(u64 (&x)[Sh::E], u64 *s, u32 tid, u32 m, const ulonglong2 *tw,
                                           const PrimeConst &pc, std::integer_sequence<int, Q...>)
{
    (inv_round<Sh, Sh::NROUND - 1 - Q>(x, s, tid, m, tw, pc), ...);
}

// Inverse negacyclic NTT (with N^-1) of one limb. If the caller already
// holds the block's values in x[] in last_pos order, pass HAVE_X = true and
// load is not called; otherwise load(P) gives the NTT-domain value at
// position P (below 4p). store(P, v) receives the canonical coefficient P.
template <class Sh, bool HAVE_X, class Load, class Store>
__device__ __forceinline__ void ntt_inv_block(u64 *s, u32 m, u32 rbase, const ulonglong2 *tw, const PrimeConst &pc,
                                              Load load, Store store, u64 (&x)[Sh::E])
{
    const u32 tid = thread_index<Sh::T>();
    if constexpr (!HAVE_X) {
#pragma unroll
        for (int e = 0; e < Sh::E; e++) x[e] = load(last_pos<Sh>(m, tid, e));
    }
    inv_rounds<Sh>(x, s, tid, m, tw, pc, std::make_integer_sequence<int, Sh::NROUND>{});
    using R0 = RoundOf<Sh, 0>;
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
        constexpr int COLS = Sh::E / (int)C;
        const u32 s_base = smem_u32(s);
        u64 fold = 0;   // every word read from the peers, for the final barrier
#pragma unroll
        for (int c = 0; c < COLS; c++) {
            const int j = (int)(m * (Sh::B / C)) + c * (int)Sh::T + (int)tid;
            const u32 a = s_base + swz<Sh::LOG_E>((u32)j) * 8u;
            u64 v[C];
#pragma unroll
            for (u32 t = 0; t < C; t++) v[t] = ld_cluster(map_to_rank(a, rbase + t));
#pragma unroll
            for (u32 t = 0; t < C; t++) fold |= v[t];
#pragma unroll
            for (int SS = 0; SS < Sh::LOG_C; SS++) {
                const int S = Sh::LOG_C - 1 - SS;
                const u32 half = C >> (S + 1);
                ulonglong2 ws[C / 2];   // this stage's twiddles only
                if (S > 0) {
#pragma unroll
                    for (int g = 0; g < (1 << S); g++) ws[g] = ld_tw(tw, inv_tw_pos(Sh::LOG_N, S, g));
                }
#pragma unroll
                for (u32 t = 0; t < C; t++) {
                    if (t & half) continue;
                    if (S == 0) {
                        gs_last(v[t], v[t + half], pc);
                    } else {
                        const ulonglong2 w = ws[t >> (Sh::LOG_C - S)];
                        gs_butterfly(v[t], v[t + half], w.x, w.y, pc);
                    }
                }
            }
#pragma unroll
            for (u32 t = 0; t < C; t++) store((int)t * (int)Sh::B + j, v[t]);
        }
        // peers may still read this CTA's shared memory; the arrive waits
        // for this thread's own remote reads (the fold), also where the
        // stores are switched off
        cluster_sync_war_fold(fold);
    }
}

}  // namespace he
