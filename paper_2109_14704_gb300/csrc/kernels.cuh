// kernels.cuh -- the CUDA kernels of the library, as templates over the NTT
// shape (words per CTA, CTAs per cluster). inst_n*.cu instantiate them per
// polynomial degree; launch.h describes the host-side launchers.
#pragma once
#include <stdint.h>

#include "launch.h"
#include "ntt_core.cuh"

namespace he {

// ============================================================ plain NTT ====

// Bulk tensor store of the forward transform's output (one warp, 16 words
// a thread: thread l of warp w holds the 16 words of row row0 + 32 w + l of
// the tensor map's view, rows of 128 bytes). The warp's rows of the shared
// block are its own from the last exchange on (each thread read back only
// its own row), so it stages them there: 16-byte chunk c of a row goes to
// chunk c ^ (bits 7..9 of the row's address), the 128-byte swizzle, which
// keeps every group of eight lanes on distinct banks. Then one lane issues
// the 4 KB store and waits until it has read the rows (the block is not
// touched again). Against four 256-bit stores a lane, each warp store
// touching 32 lines, the rows leave through the copy engine: measured 1 %
// off the forward transform at N = 2^15.
__device__ __forceinline__ void tma_store_rows(const u64 (&x)[16], u32 wbase, const CUtensorMap *tm, u32 row)
{
    const u32 lane = threadIdx.x & 31u;
    const u32 ra = wbase + lane * 128u;
    const u32 sw = (ra >> 7) & 7u;
#pragma unroll
    for (int c = 0; c < 8; c++)
        asm volatile("st.shared.v2.u64 [%0], {%1, %2};" ::"r"(ra + ((c ^ sw) << 4)), "l"(x[2 * c]), "l"(x[2 * c + 1])
                     : "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // visible to the copy engine
    __syncwarp();
    if (lane == 0) {
        asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];"
                     ::"l"(tm), "r"(0), "r"(row), "r"(wbase) : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncwarp();
}

// Forward or inverse transform of one limb stored at `data` (in place). The
// forward transform's last round and the inverse transform's first round
// give each thread runs of consecutive words, which move as 32-byte quarters
// (streaming cache hints: every word is read and written once per launch);
// the cross-CTA columns move as single coalesced words. Stores are skipped
// when !valid (idle sub-clusters of the mixed-degree kernel). With a tensor
// map tm (forward, 16 words a thread, the limb block's first row row0) the
// output leaves by bulk tensor stores instead, where the warp's rows in
// shared memory are 1024-byte aligned (the swizzle's period).
template <class Sh, bool INV>
__device__ __forceinline__ void ntt_limb(u64 *smem, u32 m, u32 rbase, u64 *data, const ulonglong2 *tw,
                                         const PrimeConst &pc, bool valid = true, const CUtensorMap *tm = nullptr,
                                         u32 row0 = 0)
{
    u64 x[Sh::E];
    const u32 tid = threadIdx.x;
    if constexpr (!INV) {
        auto ld = [&](int P) -> u64 { return __ldcs(reinterpret_cast<const unsigned long long *>(data + P)); };
        auto nost = [&](u32, u64) {};
        ntt_fwd_block<Sh>(smem, m, rbase, tw, pc, ld, nost, x);
        if constexpr (Sh::E == 16) {
            const u32 wbase = smem_u32(smem) + (tid >> 5) * 4096u;
            if (tm && valid && (wbase & 1023u) == 0) {
                tma_store_rows(x, wbase, tm, row0 + (tid >> 5) * 32u);
                return;
            }
        }
        if (valid) {
#pragma unroll
            for (int e = 0; e < Sh::E; e += 4)
                st4_cs(data + last_pos<Sh>(m, tid, e), x[e], x[e + 1], x[e + 2], x[e + 3]);
        }
    } else {
#pragma unroll
        for (int e = 0; e < Sh::E; e += 4)
            ld4_cs(data + last_pos<Sh>(m, tid, e), x[e], x[e + 1], x[e + 2], x[e + 3]);
        auto nold = [&](u32) -> u64 { return 0; };
        auto st = [&](int P, u64 v) {
            if (valid) __stcs(reinterpret_cast<unsigned long long *>(data + P), (unsigned long long)v);
        };
        ntt_inv_block<Sh, true>(smem, m, rbase, tw, pc, nold, st, x);
    }
}

template <class Sh, bool INV>
__device__ __forceinline__ void resolve_item(const NttLaunch &a, u32 item, u64 *&data, const ulonglong2 *&tw,
                                             const PrimeConst *&pcp)
{
    if (a.jobs) {
        const LimbJob &j = a.jobs[item];
        data = j.data;
        tw = INV ? j.tw_inv : j.tw_fwd;
        pcp = j.pc;
    } else {
        data = a.base + (size_t)item * Sh::N;
        const u32 pr = a.first_prime + item % a.limbs;
        tw = (INV ? a.tw_inv : a.tw_fwd) + (size_t)pr * Sh::N;
        pcp = a.pc + pr;
    }
}

// Ask L2 for this CTA's block (B words at m B) of limb `item` of the batch,
// if it exists: one bulk prefetch issued by one thread, no registers held
// and nothing waited for. Limbs read later by other clusters then come from
// L2 instead of HBM, which hides the first-stage load latency.
template <class Sh>
__device__ __forceinline__ void prefetch_limb_block(const NttLaunch &a, u32 item, u32 m)
{
    if (threadIdx.x != 0 || item >= a.items) return;
    const u64 *p = a.jobs ? a.jobs[item].data : a.base + (size_t)item * Sh::N;
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p + (size_t)m * Sh::B), "r"(Sh::B * 8u)
                 : "memory");
}

// One cluster per limb. With a.prefetch = the number of co-resident
// clusters, limb item + a.prefetch is the one a cluster started about one
// limb-time from now will take.
template <int LOG_B, int LOG_C, int LOG_E, bool INV, int OCC = 0>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E, OCC>::MIN_CTAS)
k_ntt(const __grid_constant__ NttLaunch a)   // grid constant: tmap is addressed in place
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(1024) u64 smem[];
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 item = blockIdx.x >> LOG_C;
    if (a.prefetch) prefetch_limb_block<Sh>(a, item + a.prefetch, m);
    u64 *data;
    const ulonglong2 *tw;
    const PrimeConst *pcp;
    resolve_item<Sh, INV>(a, item, data, tw, pcp);
    const PrimeConst pc = *pcp;
    if (!INV && a.tma_store)
        ntt_limb<Sh, INV>(smem, m, 0, data, tw, pc, true, &a.tmap, (u32)(((size_t)item * Sh::N + m * Sh::B) >> 4));
    else
        ntt_limb<Sh, INV>(smem, m, 0, data, tw, pc);
}

// Persistent form: a fixed grid of clusters walks the limbs (job list or
// uniform batch).
template <int LOG_B, int LOG_C, int LOG_E, bool INV, int OCC = 0>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E, OCC>::MIN_CTAS)
k_ntt_persistent(NttLaunch a)
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(16) u64 smem[];
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 clusters = gridDim.x >> LOG_C;
    bool first = true;
    for (u32 item = blockIdx.x >> LOG_C; item < a.items; item += clusters) {
        if (!first) ntt_barrier<Sh>();
        first = false;
        if (a.prefetch) prefetch_limb_block<Sh>(a, item + clusters, m);   // this cluster's next limb
        u64 *data;
        const ulonglong2 *tw;
        const PrimeConst *pcp;
        resolve_item<Sh, INV>(a, item, data, tw, pcp);
        const PrimeConst pc = *pcp;
        ntt_limb<Sh, INV>(smem, m, 0, data, tw, pc);
    }
}

// Mixed-degree form: clusters of 8 CTAs of 2^12 words each take units of a
// list (plans launch one cluster per unit; a smaller grid walks the list); a
// unit of degree 2^(12+c) holds up to 8 >> c limbs, each transformed by a
// sub-cluster of 2^c CTAs (cluster ranks rbase .. rbase + 2^c - 1). One
// launch covers every degree from 2^12 to 2^15. Sub-clusters without a limb
// in the last unit of a degree recompute the unit's first limb with stores
// switched off, so that every CTA of the cluster passes the same cluster
// barriers. Not inlined: each shape gets its own register allocation (one
// kernel body holding all four shapes spilled up to 656 bytes at 64
// registers; this way 12-44 bytes, 172 for the smallest inverse).
template <class Sh, bool INV>
__device__ __noinline__ void mixed_unit(u64 *smem, u32 rank, const MixedUnit &un, const LimbJob *jobs)
{
    if constexpr (Sh::LOG_C == 3) {
        // the whole cluster transforms the unit's one limb
        const LimbJob j = jobs[un.first_job];
        const PrimeConst pc = *j.pc;
        ntt_limb<Sh, INV>(smem, rank, 0, j.data, INV ? j.tw_inv : j.tw_fwd, pc);
    } else if constexpr (Sh::LOG_C == 0) {
        // one CTA per limb and no cluster barrier inside the transform: a
        // CTA without a limb has nothing to do
        if (rank >= un.n_jobs) return;
        const LimbJob j = jobs[un.first_job + rank];
        const PrimeConst pc = *j.pc;
        ntt_limb<Sh, INV>(smem, 0, 0, j.data, INV ? j.tw_inv : j.tw_fwd, pc);
    } else {
        const u32 sub = rank >> Sh::LOG_C;
        const u32 m = rank & (Sh::C - 1);
        const u32 rbase = sub << Sh::LOG_C;
        const bool valid = sub < un.n_jobs;
        const LimbJob j = jobs[un.first_job + (valid ? sub : 0u)];
        const PrimeConst pc = *j.pc;
        ntt_limb<Sh, INV>(smem, m, rbase, j.data, INV ? j.tw_inv : j.tw_fwd, pc, valid);
    }
}

template <bool INV>
__global__ void __launch_bounds__(256, 4) k_ntt_mixed(const MixedUnit *units, u32 n_units, const LimbJob *jobs)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 rank = cluster_ctarank();
    const u32 clusters = gridDim.x >> 3;
    bool first = true;
    for (u32 ui = blockIdx.x >> 3; ui < n_units; ui += clusters) {
        if (!first) cluster_sync_war();
        first = false;
        const MixedUnit un = units[ui];
        switch (un.log_n) {
        case 12: mixed_unit<NttShape<12, 0>, INV>(smem, rank, un, jobs); break;
        case 13: mixed_unit<NttShape<12, 1>, INV>(smem, rank, un, jobs); break;
        case 14: mixed_unit<NttShape<12, 2>, INV>(smem, rank, un, jobs); break;
        default: mixed_unit<NttShape<12, 3>, INV>(smem, rank, un, jobs); break;
        }
    }
}

// ============================================================ fused product

// c = a b mod (X^N + 1, q) for one limb per cluster (Sec. II-B: the
// product of two polynomials is the inverse transform of the pointwise
// product of their transforms): the forward transform of a, its values
// parked in a second shared-memory block (each thread its own positions),
// the forward transform of b, the pointwise Barrett product in registers,
// and the inverse transform straight to c. Per word 16 B are read and 8 B
// written, against 72 B for three separate passes.
template <int LOG_B, int LOG_C, int LOG_E>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::NEGA_MIN_CTAS)
k_negacyclic(NegaLaunch a)
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(16) u64 smem[];
    u64 *park = smem + Sh::B;                    // [E][T]
    const u32 tid = threadIdx.x;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 item = blockIdx.x >> LOG_C;
    const u32 pr = item % a.limbs;
    const PrimeConst pc = a.pc[pr];
    const ulonglong2 *twf = a.tw_fwd + (size_t)pr * Sh::N, *twi = a.tw_inv + (size_t)pr * Sh::N;
    const u64 *A = a.a + (size_t)item * Sh::N, *Bp = a.b + (size_t)item * Sh::N;
    u64 *C = a.c + (size_t)item * Sh::N;
    u64 x[Sh::E];
    auto nost = [&](u32, u64) {};
    // one copy of the forward transform run twice (a loop, not unrolled):
    // two inlined copies let the compiler keep the first one's address and
    // twiddle values live into the second, which spills
#pragma unroll 1
    for (int it = 0; it < 2; it++) {
        const u64 *src = it ? Bp : A;
        if (it) ntt_barrier<Sh>();
        auto ld = [&](int P) -> u64 { return __ldcs(reinterpret_cast<const unsigned long long *>(src + P)); };
        ntt_fwd_block<Sh>(smem, m, 0, twf, pc, ld, nost, x);
        if (it == 0) {
#pragma unroll
            for (int e = 0; e < Sh::E; e++) park[e * Sh::T + tid] = x[e];
        } else {
#pragma unroll
            for (int e = 0; e < Sh::E; e++) x[e] = mul_mod(x[e], park[e * Sh::T + tid], pc);
        }
    }
    ntt_barrier<Sh>();
    auto nold = [&](u32) -> u64 { return 0; };
    auto st = [&](int P, u64 v) { __stcs(reinterpret_cast<unsigned long long *>(C + P), (unsigned long long)v); };
    ntt_inv_block<Sh, true>(smem, m, 0, twi, pc, nold, st, x);
}

#ifdef HE_MISC_KERNELS  // defined by the one translation unit that owns them
// ======================================================== naive radix-2 ====
// The baseline of Sec. III-B: one launch per stage, each thread one
// butterfly, data exchanged through global memory, and a final pass that
// reduces the lazy range to [0, p) (forward) -- 2 N log N + 2 N global
// accesses.

__global__ void k_ntt_naive_stage(NttLaunch a, u32 log_n, u32 S, bool inv)
{
    const u32 N = 1u << log_n;
    const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const size_t total = (size_t)a.items * (N / 2);
    if (gid >= total) return;
    const u32 item = (u32)(gid / (N / 2));
    const u32 b = (u32)(gid % (N / 2));
    u64 *data = a.base + (size_t)item * N;
    const u32 pr = a.first_prime + item % a.limbs;
    const PrimeConst pc = a.pc[pr];
    const u32 t = N >> (S + 1);
    const u32 g = b / t;
    const u32 j = 2 * g * t + (b % t);
    u64 x = data[j], y = data[j + t];
    if (!inv) {
        const ulonglong2 w = a.tw_fwd[(size_t)pr * N + (1u << S) + g];
        ct_butterfly(x, y, w.x, w.y, pc);
    } else if (S == 0) {
        gs_last(x, y, pc);
    } else {
        const ulonglong2 w = a.tw_inv[(size_t)pr * N + inv_tw_pos((int)log_n, (int)S, (int)g)];
        gs_butterfly(x, y, w.x, w.y, pc);
    }
    data[j] = x;
    data[j + t] = y;
}

__global__ void k_ntt_naive_final(NttLaunch a, u32 log_n)
{
    const u32 N = 1u << log_n;
    const size_t gid = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (size_t)a.items * N) return;
    const u32 item = (u32)(gid >> log_n);
    const PrimeConst &pc = a.pc[a.first_prime + item % a.limbs];
    u64 v = a.base[gid];
    a.base[gid] = reduce_from_fwd_range(v, pc);
}

// =========================================================== dyadic ========

// out = a * b mod q for `items` limbs of N words; 2 words per thread.
__global__ void k_dyadic(u64 *out, const u64 *a, const u64 *b, u32 log_n, u32 items, u32 limbs,
                         u32 first_prime, const PrimeConst *pcs)
{
    const size_t total2 = ((size_t)items << log_n) >> 1;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total2;
         g += (size_t)gridDim.x * blockDim.x) {
        const size_t e = g * 2;
        const u32 item = (u32)(e >> log_n);
        const PrimeConst pc = pcs[first_prime + item % limbs];
        const ulonglong2 va = *reinterpret_cast<const ulonglong2 *>(a + e);
        const ulonglong2 vb = *reinterpret_cast<const ulonglong2 *>(b + e);
        ulonglong2 r;
        r.x = mul_mod(va.x, vb.x, pc);
        r.y = mul_mod(va.y, vb.y, pc);
        *reinterpret_cast<ulonglong2 *>(out + e) = r;
    }
}

// ============================================================ Mul ==========

// out3[c] = (a0 b0, a0 b1 + a1 b0, a1 b1) per limb (Sec. II-A), count pairs.
__global__ void k_tensor(u64 *out3, const u64 *ct_a, const u64 *ct_b, u32 log_n, u32 n, u32 count,
                         const PrimeConst *pcs)
{
    const size_t per = (size_t)n << log_n;           // words per component
    const size_t total2 = (size_t)count * per / 2;
    for (size_t g = (size_t)blockIdx.x * blockDim.x + threadIdx.x; g < total2;
         g += (size_t)gridDim.x * blockDim.x) {
        const size_t e = g * 2;
        const size_t c = e / per;
        const size_t off = e - c * per;
        const u32 limb = (u32)(off >> log_n);
        const PrimeConst pc = pcs[limb];
        const u64 *A = ct_a + c * 2 * per + off;
        const u64 *Bp = ct_b + c * 2 * per + off;
        const ulonglong2 a0 = *reinterpret_cast<const ulonglong2 *>(A);
        const ulonglong2 a1 = *reinterpret_cast<const ulonglong2 *>(A + per);
        const ulonglong2 b0 = *reinterpret_cast<const ulonglong2 *>(Bp);
        const ulonglong2 b1 = *reinterpret_cast<const ulonglong2 *>(Bp + per);
        u64 *O = out3 + c * 3 * per + off;
        ulonglong2 d0, d1, d2;
        d0.x = mul_mod(a0.x, b0.x, pc);
        d0.y = mul_mod(a0.y, b0.y, pc);
        d1.x = mad2_mod(a0.x, b1.x, a1.x, b0.x, pc);
        d1.y = mad2_mod(a0.y, b1.y, a1.y, b0.y, pc);
        d2.x = mul_mod(a1.x, b1.x, pc);
        d2.y = mul_mod(a1.y, b1.y, pc);
        *reinterpret_cast<ulonglong2 *>(O) = d0;
        *reinterpret_cast<ulonglong2 *>(O + per) = d1;
        *reinterpret_cast<ulonglong2 *>(O + 2 * per) = d2;
    }
}

// ct_out = ct_a + ct_b mod q per limb, `words` words of ciphertexts with n
// limbs of 2^log_n words (any number of components), two words per thread.
__global__ void k_ct_add(u64 *out, const u64 *a, const u64 *b, u64 words, u32 log_n, u32 n, const PrimeConst *pcs)
{
    for (u64 g = (u64)blockIdx.x * blockDim.x + threadIdx.x; 2 * g < words; g += (u64)gridDim.x * blockDim.x) {
        const u64 e = 2 * g;
        const PrimeConst pc = pcs[(u32)((e >> log_n) % n)];
        const ulonglong2 x = *reinterpret_cast<const ulonglong2 *>(a + e);
        const ulonglong2 y = *reinterpret_cast<const ulonglong2 *>(b + e);
        *reinterpret_cast<ulonglong2 *>(out + e) = make_ulonglong2(add_mod(x.x, y.x, pc.p), add_mod(x.y, y.y, pc.p));
    }
}

// The automorphism X -> X^g (g odd) on NTT-domain polynomials of 2^log_n
// words (any number of them, back to back). Output index i holds
// a(psi^(2 brv(i) + 1)) (the order of he_ntt_fwd), so the image
// sigma(a)(psi^(2 brv(i) + 1)) = a(psi^(g (2 brv(i) + 1))) is the input
// word at index brv((g (2 brv(i) + 1) mod 2N - 1) / 2): a gather within
// each polynomial, the same for every limb.
__global__ void k_ct_automorph(u64 *out, const u64 *in, u64 words, u32 log_n, u32 g)
{
    const u32 N = 1u << log_n, mask2 = 2 * N - 1, sh = 32 - log_n;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < words; e += (u64)gridDim.x * blockDim.x) {
        const u32 i = (u32)e & (N - 1);
        const u32 r = __brev(i) >> sh;
        const u32 t = (u32)(((u64)g * (2 * r + 1)) & mask2);
        const u32 src = __brev((t - 1) >> 1) >> sh;
        out[e] = __ldg(reinterpret_cast<const unsigned long long *>(in + (e - i) + src));
    }
}

// ============================================ encrypted matrix product ======
// Tensor part of C += A B (Sec. IV-E matMul_mxnxk; Sec. II-A Mul): for each
// limb and position, T[i][j] = sum_l (a0 b0, a0 b1 + a1 b0, a1 b1) over the
// pairs (A[i][l], B[l][j]) mod q. For q >= 2^32 the 128-bit products are
// summed without reduction (a0 b1 + a1 b0 included: the fused
// multiply-add of Sec. III-A-1 carried over the whole sum) and reduced once
// per 32 terms; smaller moduli reduce every term (Barrett, one reduction for
// a0 b1 + a1 b0). A thread owns one limb, two positions, row i and MM_TJ
// consecutive output columns, so each A word it loads serves MM_TJ products;
// consecutive threads take consecutive positions (coalesced 16-byte loads).
constexpr u32 MM_TJ = 2;

// (h, lo) += a b as a 128-bit sum.
__device__ __forceinline__ void mac128(u64 &h, u64 &lo, u64 a, u64 b)
{
    const u64 pl = a * b, ph = __umul64hi(a, b);
    lo += pl;
    h += ph + (lo < pl ? 1 : 0);
}

__global__ void k_ct_matmul_tensor(u64 *t, const u64 *a, const u64 *b, u32 m, u32 k, u32 n, u32 log_n, u32 limbs,
                                   const PrimeConst *pcs)
{
    const u32 half = 1u << (log_n - 1);
    const u32 jt_count = (n + MM_TJ - 1) / MM_TJ;
    const size_t poly = (size_t)limbs << log_n;             // words per component
    const u64 total = (u64)m * jt_count * limbs * half;
    for (u64 q = (u64)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (u64)gridDim.x * blockDim.x) {
        const u32 P = (u32)(q % half) * 2;
        const u32 limb = (u32)((q / half) % limbs);
        const u32 jt = (u32)((q / ((u64)half * limbs)) % jt_count);
        const u32 i = (u32)(q / ((u64)half * limbs * jt_count));
        const PrimeConst pc = pcs[limb];
        const size_t off = ((size_t)limb << log_n) + P;
        u64 acc[MM_TJ][3][2];
#pragma unroll
        for (u32 jj = 0; jj < MM_TJ; jj++)
#pragma unroll
            for (int c = 0; c < 3; c++) acc[jj][c][0] = acc[jj][c][1] = 0;
        if (pc.p >= (1ull << 32)) {
            // lazy: 128-bit sums of up to 64 products (< 2^126), reduced per
            // chunk of 32 terms: hi mod p, then hi 2^64 + lo = hi c64 + lo
            const u64 c64 = barrett_reduce(1, 0, pc.p, pc.mu, pc.bits);   // 2^64 mod p
            for (u32 l0 = 0; l0 < k; l0 += 32) {
                u64 h[MM_TJ][3][2], lo[MM_TJ][3][2];
#pragma unroll
                for (u32 jj = 0; jj < MM_TJ; jj++)
#pragma unroll
                    for (int c = 0; c < 3; c++) h[jj][c][0] = h[jj][c][1] = lo[jj][c][0] = lo[jj][c][1] = 0;
                const u32 l1 = min(k, l0 + 32);
                for (u32 l = l0; l < l1; l++) {
                    const u64 *ap = a + ((size_t)i * k + l) * 2 * poly + off;
                    const ulonglong2 a0 = __ldg(reinterpret_cast<const ulonglong2 *>(ap));
                    const ulonglong2 a1 = __ldg(reinterpret_cast<const ulonglong2 *>(ap + poly));
#pragma unroll
                    for (u32 jj = 0; jj < MM_TJ; jj++) {
                        const u32 j = jt * MM_TJ + jj;
                        if (j >= n) break;
                        const u64 *bp = b + ((size_t)l * n + j) * 2 * poly + off;
                        const ulonglong2 b0 = __ldg(reinterpret_cast<const ulonglong2 *>(bp));
                        const ulonglong2 b1 = __ldg(reinterpret_cast<const ulonglong2 *>(bp + poly));
                        mac128(h[jj][0][0], lo[jj][0][0], a0.x, b0.x);
                        mac128(h[jj][0][1], lo[jj][0][1], a0.y, b0.y);
                        mac128(h[jj][1][0], lo[jj][1][0], a0.x, b1.x);
                        mac128(h[jj][1][0], lo[jj][1][0], a1.x, b0.x);
                        mac128(h[jj][1][1], lo[jj][1][1], a0.y, b1.y);
                        mac128(h[jj][1][1], lo[jj][1][1], a1.y, b0.y);
                        mac128(h[jj][2][0], lo[jj][2][0], a1.x, b1.x);
                        mac128(h[jj][2][1], lo[jj][2][1], a1.y, b1.y);
                    }
                }
#pragma unroll
                for (u32 jj = 0; jj < MM_TJ; jj++)
#pragma unroll
                    for (int c = 0; c < 3; c++)
#pragma unroll
                        for (int x = 0; x < 2; x++) {
                            const u64 r1 = barrett_reduce(0, h[jj][c][x], pc.p, pc.mu, pc.bits);
                            u64 zh, zl;
                            mul_wide(r1, c64, zh, zl);
                            zl += lo[jj][c][x];
                            zh += (zl < lo[jj][c][x]) ? 1 : 0;
                            acc[jj][c][x] = add_mod(acc[jj][c][x], barrett_reduce(zh, zl, pc.p, pc.mu, pc.bits), pc.p);
                        }
            }
        } else
        for (u32 l = 0; l < k; l++) {
            const u64 *ap = a + ((size_t)i * k + l) * 2 * poly + off;
            const ulonglong2 a0 = __ldg(reinterpret_cast<const ulonglong2 *>(ap));
            const ulonglong2 a1 = __ldg(reinterpret_cast<const ulonglong2 *>(ap + poly));
#pragma unroll
            for (u32 jj = 0; jj < MM_TJ; jj++) {
                const u32 j = jt * MM_TJ + jj;
                if (j >= n) break;
                const u64 *bp = b + ((size_t)l * n + j) * 2 * poly + off;
                const ulonglong2 b0 = __ldg(reinterpret_cast<const ulonglong2 *>(bp));
                const ulonglong2 b1 = __ldg(reinterpret_cast<const ulonglong2 *>(bp + poly));
                acc[jj][0][0] = add_mod(acc[jj][0][0], mul_mod(a0.x, b0.x, pc), pc.p);
                acc[jj][0][1] = add_mod(acc[jj][0][1], mul_mod(a0.y, b0.y, pc), pc.p);
                acc[jj][1][0] = add_mod(acc[jj][1][0], mad2_mod(a0.x, b1.x, a1.x, b0.x, pc), pc.p);
                acc[jj][1][1] = add_mod(acc[jj][1][1], mad2_mod(a0.y, b1.y, a1.y, b0.y, pc), pc.p);
                acc[jj][2][0] = add_mod(acc[jj][2][0], mul_mod(a1.x, b1.x, pc), pc.p);
                acc[jj][2][1] = add_mod(acc[jj][2][1], mul_mod(a1.y, b1.y, pc), pc.p);
            }
        }
#pragma unroll
        for (u32 jj = 0; jj < MM_TJ; jj++) {
            const u32 j = jt * MM_TJ + jj;
            if (j >= n) break;
            u64 *tp = t + ((size_t)i * n + j) * 3 * poly + off;
#pragma unroll
            for (int c = 0; c < 3; c++)
                *reinterpret_cast<ulonglong2 *>(tp + c * poly) = make_ulonglong2(acc[jj][c][0], acc[jj][c][1]);
        }
    }
}

// ============================================================ Encrypt ======

// Residues of the encryption's small random polynomials: out[c][w][l][i] =
// src_w[c][i] mod q_l for w = 0, 1, 2 (v, e0, e1; signed 8-bit values with
// |x| < q), count messages of n limbs.
__global__ void k_enc_noise(u64 *out, const int8_t *v, const int8_t *e0, const int8_t *e1, u32 log_n, u32 n,
                            u32 count, const PrimeConst *pcs)
{
    const u64 N = 1ull << log_n, words = (u64)count * 3 * n * N;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < words; e += (u64)gridDim.x * blockDim.x) {
        const u64 i = e & (N - 1), row = e >> log_n;
        const u32 l = (u32)(row % n), w = (u32)((row / n) % 3);
        const u64 c = row / (3 * (u64)n);
        const int8_t *src = w == 0 ? v : (w == 1 ? e0 : e1);
        const int x = src[c * N + i];
        out[e] = x >= 0 ? (u64)x : pcs[l].p - (u64)(-x);
    }
}

// Randomness of encryption drawn on the device (Sec. II-A Encrypt: a
// uniform ternary mask v and Gaussian-like errors e0, e1). Generator:
// SplitMix64 in counter form (Steele, Lea and Flood 2014): output k of the
// stream with key `seed` is mix(seed + (k + 1) * 0x9E3779B97F4A7C15), with
// mix(z): z = (z ^ z >> 30) * 0xBF58476D1CE4E5B9; z = (z ^ z >> 27) *
// 0x94D049BB133111EB; z ^ z >> 31. Draw w (0: v, 1: e0, 2: e1) of message c
// at coefficient i uses output k = (3 c + w) N + i:
//   v  = (r mod 3) - 1                        (bias below 2^-63)
//   e  = popcount(r & (2^20 - 1)) - popcount((r >> 20) & (2^20 - 1)),
// the centred binomial distribution of parameter 20 (variance 10, standard
// deviation 3.16, |e| <= 20): integer-only, so that any implementation
// following this definition reproduces the draws bit for bit.
__device__ __forceinline__ u64 splitmix64_at(u64 seed, u64 k)
{
    u64 z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ int enc_draw(u64 seed, u32 w, u64 c, u64 i, u32 log_n)
{
    const u64 r = splitmix64_at(seed, ((3 * c + w) << log_n) + i);
    if (w == 0) return (int)(r % 3u) - 1;
    return __popcll(r & 0xFFFFFull) - __popcll((r >> 20) & 0xFFFFFull);
}

// The draws themselves, as signed 8-bit values [count][N] each.
__global__ void k_enc_draws(int8_t *v, int8_t *e0, int8_t *e1, u64 seed, u32 log_n, u32 count)
{
    const u64 N = 1ull << log_n, total = (u64)count * N;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u64 c = e >> log_n, i = e & (N - 1);
        v[e] = (int8_t)enc_draw(seed, 0, c, i, log_n);
        e0[e] = (int8_t)enc_draw(seed, 1, c, i, log_n);
        e1[e] = (int8_t)enc_draw(seed, 2, c, i, log_n);
    }
}

// As k_enc_noise, with the draws generated in place from the seed.
__global__ void k_enc_noise_seeded(u64 *out, u64 seed, u32 log_n, u32 n, u32 count, const PrimeConst *pcs)
{
    const u64 N = 1ull << log_n, words = (u64)count * 3 * n * N;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < words; e += (u64)gridDim.x * blockDim.x) {
        const u64 i = e & (N - 1), row = e >> log_n;
        const u32 l = (u32)(row % n), w = (u32)((row / n) % 3);
        const u64 c = row / (3 * (u64)n);
        const int x = enc_draw(seed, w, c, i, log_n);
        out[e] = x >= 0 ? (u64)x : pcs[l].p - (u64)(-x);
    }
}

// Public-key encryption (Sec. II-A) from the transformed randomness:
// c0 = v pk0 + pt + e0, c1 = v pk1 + e1 (NTT domain, limb by limb).
// noise [count][3][n][N] (v, e0, e1 transformed), pt [count][n][N],
// pk [2][pk_limbs][N], ct [count][2][n][N].
__global__ void k_enc_combine(u64 *ct, const u64 *noise, const u64 *pt, const u64 *pk, u32 log_n, u32 n, u32 count,
                              u32 pk_limbs, const PrimeConst *pcs)
{
    const u64 N = 1ull << log_n, per = (u64)n * N, total = (u64)count * per;
    for (u64 e = (u64)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (u64)gridDim.x * blockDim.x) {
        const u64 c = e / per, off = e - c * per;
        const u32 l = (u32)(off >> log_n);
        const PrimeConst pc = pcs[l];
        const u64 *z = noise + c * 3 * per + off;
        const u64 vh = z[0], e0h = z[per], e1h = z[2 * per];
        const u64 c0 = add_mod(add_mod(mul_mod(vh, pk[off], pc), pt[e], pc.p), e0h, pc.p);
        const u64 c1 = add_mod(mul_mod(vh, pk[(u64)pk_limbs * N + off], pc), e1h, pc.p);
        ct[c * 2 * per + off] = c0;
        ct[c * 2 * per + per + off] = c1;
    }
}
#endif  // HE_MISC_KERNELS

// ============================================== key switching and rescale ==
//
// Relin (Sec. II-A) with RNS digits and one special prime P, as four kernels
// over all ciphertexts of a batch:
//   k_ks_digits   INTT_{q_j}(c[2]_j) -> coefficient digits c2_j     (n INTT)
//   k_ks_modup    for each target t in {q_0..q_l, P}:
//                 acc_k[t] = sum_j NTT_t(c2_j mod t) * evk[j][k][t]  (n^2 NTT)
//                 (for t = q_j the NTT-domain c[2]_j is used as is); on P the
//                 accumulators are brought back by INTT_P and kept as the
//                 coefficient-domain residues y_k = [x_k]_P          (2 INTT);
//                 on the data primes the stored accumulator already holds
//                 d_k P + acc_k, so that the mod-down needs no d_k:
//   k_ks_moddown  out_k[i] = d_k[i] + (acc_k[q_i] - NTT(r_k mod q_i)) P^-1
//                          = (stored acc - NTT(r_k mod q_i)) P^-1,
//                 r_k the centred lift of y_k                        (2n NTT)
// RS (Sec. II-A): k_rs_lift brings c_k[q_l] to the coefficient domain
// (2 INTT), k_rs combines (c_k[q_i] - NTT(r mod q_i)) q_l^-1 (2(n-1) NTT).
// MulLinRS fuses Mul into the loads and the mod-down of limb q_l with RS's
// INTT (k_mrr_last), and mod-down with RS for the other limbs (k_mrr_rest_z,
// k_mrr_rest_out).

// Centred residue of y in [0, m) (|r| <= (m-1)/2) reduced mod q:
// y mod q, or y mod q - m mod q when y > (m-1)/2 (any word y).
__device__ __forceinline__ u64 centred_mod(u64 y, u64 half_m, u64 m_mod_q, const PrimeConst &pc)
{
    const u64 r = reduce_word_canon(y, pc);
    return y > half_m ? sub_mod(r, m_mod_q, pc.p) : r;
}

// a - x + 12p: congruent to a - x mod p and positive for a < 2^63 - 12p and
// x < 12p (a lazy forward-transform output, see ntt_fwd_block with CANON =
// false); below 2^64 for a < 2p, so it can go straight into mul_shoup.
__device__ __forceinline__ u64 lazy_sub(u64 a, u64 x, u64 twelve_p) { return a + twelve_p - x; }

// Epilogue of a lazy forward transform (ntt_fwd_block with CANON = false):
//   r(e) = (src[P] - x[e]) C mod p,  P = last_pos(e),  C' = Shoup(C),
// for every word the thread holds, into x. Positions e .. e + 3 (e = 0 mod
// 4) of the last round are consecutive and 32-byte aligned, so src moves in
// 32-byte quarters, all of them loaded before the caller stores anything
// (src may be the output: with alternating loads and stores each store
// would evict lines the next loads need).
template <class Sh>
__device__ __forceinline__ void sub_scale_run(u64 (&x)[Sh::E], const u64 *src, u64 C, u64 C_sh,
                                              const PrimeConst &pc, u32 m, u32 tid)
{
    const u64 twelve_p = 3 * pc.four_p;
    u64 v[Sh::E];
#pragma unroll
    for (int e = 0; e < Sh::E; e += 4) ld4(src + last_pos<Sh>(m, tid, e), v[e], v[e + 1], v[e + 2], v[e + 3]);
#pragma unroll
    for (int e = 0; e < Sh::E; e++) x[e] = mul_shoup(lazy_sub(v[e], x[e], twelve_p), C, C_sh, pc.p);
}

// x[] to dst at the thread's last-round positions, in 32-byte quarters.
template <class Sh>
__device__ __forceinline__ void store_run(u64 *dst, const u64 (&x)[Sh::E], u32 m, u32 tid)
{
#pragma unroll
    for (int e = 0; e < Sh::E; e += 4) st4(dst + last_pos<Sh>(m, tid, e), x[e], x[e + 1], x[e + 2], x[e + 3]);
}

// Read-only load (the kernel never writes what it reads through this).
__device__ __forceinline__ u64 rd(const u64 *p) { return __ldg(reinterpret_cast<const unsigned long long *>(p)); }

// d_k[i] at position P for component k (0 or 1): from the tensor of the two
// input ciphertexts (fused Mul) or from a 3-component input.
// Job of a mixed-level batch that owns global item `item` of stage S (the
// last job whose first item is not above it): its buffers and sizes go into
// a, and the item's index within the job is returned.
__device__ __forceinline__ u32 bind_job(EvalArgs &a, const JobTable &t, int S, u32 item)
{
    u32 lo = 0, hi = t.n_jobs - 1;
    while (lo < hi) {
        const u32 mid = (lo + hi + 1) / 2;
        if (t.job[mid].begin[S] <= item) lo = mid;
        else hi = mid - 1;
    }
    const EvalJob &J = t.job[lo];
    a.ct_a = J.ct_a;
    a.ct_b = J.ct_b;
    a.ct3 = nullptr;
    a.out = J.out;
    a.c2 = J.c2;
    a.accq = J.accq;
    a.plift = J.plift;
    a.lift2 = J.lift2;
    a.mx = J.mx;
    a.evk = J.evk;
    a.ctx = J.ctx;
    a.n = J.n;
    a.count = J.count;
    a.c_first = 0;
    return item - J.begin[S];
}

struct DSource {
    const u64 *ct_a, *ct_b, *ct3;  // per-ciphertext bases
    size_t per;                    // n * N words per component
    __device__ __forceinline__ u64 d(int k, u32 limb, u32 log_n, u32 P, const PrimeConst &pc) const
    {
        const size_t off = ((size_t)limb << log_n) + P;
        if (ct3) return rd(ct3 + k * per + off);
        if (k == 0) return mul_mod(rd(ct_a + off), rd(ct_b + off), pc);
        if (k == 1) return mad2_mod(rd(ct_a + off), rd(ct_b + per + off), rd(ct_a + per + off), rd(ct_b + off), pc);
        return mul_mod(rd(ct_a + per + off), rd(ct_b + per + off), pc);
    }
    // d_k at the two positions P, P + 1 (P even), from 16-byte loads.
    __device__ __forceinline__ ulonglong2 d2(int k, u32 limb, u32 log_n, u32 P, const PrimeConst &pc) const
    {
        const size_t off = ((size_t)limb << log_n) + P;
        auto ld = [](const u64 *q) { return __ldg(reinterpret_cast<const ulonglong2 *>(q)); };
        if (ct3) return ld(ct3 + k * per + off);
        ulonglong2 r;
        if (k == 1) {
            const ulonglong2 a0 = ld(ct_a + off), a1 = ld(ct_a + per + off);
            const ulonglong2 b0 = ld(ct_b + off), b1 = ld(ct_b + per + off);
            r.x = mad2_mod(a0.x, b1.x, a1.x, b0.x, pc);
            r.y = mad2_mod(a0.y, b1.y, a1.y, b0.y, pc);
            return r;
        }
        const size_t o = (k == 0) ? off : per + off;
        const ulonglong2 a = ld(ct_a + o), b = ld(ct_b + o);
        r.x = mul_mod(a.x, b.x, pc);
        r.y = mul_mod(a.y, b.y, pc);
        return r;
    }
    // d_k at the four positions P .. P + 3 (P = 0 mod 4) into r[0..3], from
    // 32-byte loads.
    __device__ __forceinline__ void d4(int k, u32 limb, u32 log_n, u32 P, const PrimeConst &pc, u64 *r) const
    {
        const size_t off = ((size_t)limb << log_n) + P;
        if (ct3) {
            ld4_nc(ct3 + k * per + off, r[0], r[1], r[2], r[3]);
            return;
        }
        u64 a[4], b[4];
        if (k == 1) {
            u64 a1[4], b1[4];
            ld4_nc(ct_a + off, a[0], a[1], a[2], a[3]);
            ld4_nc(ct_b + per + off, b1[0], b1[1], b1[2], b1[3]);
            ld4_nc(ct_a + per + off, a1[0], a1[1], a1[2], a1[3]);
            ld4_nc(ct_b + off, b[0], b[1], b[2], b[3]);
#pragma unroll
            for (int i = 0; i < 4; i++) r[i] = mad2_mod(a[i], b1[i], a1[i], b[i], pc);
            return;
        }
        const size_t o = (k == 0) ? off : per + off;
        ld4_nc(ct_a + o, a[0], a[1], a[2], a[3]);
        ld4_nc(ct_b + o, b[0], b[1], b[2], b[3]);
#pragma unroll
        for (int i = 0; i < 4; i++) r[i] = mul_mod(a[i], b[i], pc);
    }
};

__device__ __forceinline__ DSource dsource(const EvalArgs &a, u32 c)
{
    DSource s;
    s.per = (size_t)a.n * a.ctx.N;
    s.ct3 = a.ct3 ? a.ct3 + (size_t)c * 3 * s.per : nullptr;
    s.ct_a = a.ct_a ? a.ct_a + (size_t)c * 2 * s.per : nullptr;
    s.ct_b = a.ct_b ? a.ct_b + (size_t)c * 2 * s.per : nullptr;
    return s;
}

// Stage bodies of the MulLinRS pipeline for one item, shared by the per-
// degree kernels (one cluster per item: m = cluster rank, rbase = 0, valid)
// and the multi-degree kernels (multi.cu: sub-clusters of 2^LOG_C CTAs at
// cluster ranks rbase .. rbase + 2^LOG_C - 1; a sub-cluster without an item
// of its own recomputes a valid one with every store switched off, so that
// all CTAs of the cluster pass the same cluster barriers).

// Digit INTT: c2[c][j] = INTT_{q_j}(d2[c][j]), item = c n + j.
template <class Sh>
__device__ __forceinline__ void ks_digits_body(const EvalArgs &a, u32 item, u32 m, u32 rbase, bool valid)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 c = item / a.n, j = item % a.n;
    const PrimeConst pc = a.ctx.pc[j];
    const DSource ds = dsource(a, c);
    u64 *out = a.c2 + ((size_t)c * a.n + j) * Sh::N;
    const u32 tid = threadIdx.x;
    u64 x[Sh::E];
    // d2 at the thread's inverse-input positions (consecutive quarters)
#pragma unroll
    for (int e = 0; e < Sh::E; e += 4) ds.d4(2, j, Sh::LOG_N, (u32)last_pos<Sh>(m, tid, e), pc, x + e);
    auto nold = [&](u32) -> u64 { return 0; };
    auto st = [&](u32 P, u64 v) {
        if (valid) out[P] = v;
    };
    ntt_inv_block<Sh, true>(smem, m, rbase, a.ctx.tw_inv + (size_t)j * Sh::N, pc, nold, st, x);
}

template <int LOG_B, int LOG_C, int LOG_E, bool JOBS = false>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::MIN_CTAS)
k_ks_digits(EvalArgs a0, JobsArg<JOBS> tab)
{
    EvalArgs a = a0;
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    u32 item = blockIdx.x >> LOG_C;
    if constexpr (JOBS) item = bind_job(a, tab, JS_DIGITS, item);
    ks_digits_body<Sh>(a, item, m, 0, true);
}

template <int LOG_B, int LOG_C, int LOG_E>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::EVAL_MIN_CTAS)
k_ks_modup(EvalArgs a)
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(16) u64 smem[];
    u64 *acc = smem + Sh::B;                   // [2][E][T], own positions only
    const u32 tid = threadIdx.x;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 item = blockIdx.x >> LOG_C;
    const u32 n = a.n;
    const u32 c = item / (n + 1), t = item % (n + 1);
    const u32 tp = (t == n) ? a.ctx.n_data : t; // prime index of the target
    const PrimeConst pc = a.ctx.pc[tp];
    const DSource ds = dsource(a, c);
    const ulonglong2 *twf = a.ctx.tw_fwd + (size_t)tp * Sh::N;
    u64 x[Sh::E];
    for (u32 j = 0; j < n; j++) {
        if (t == j) {
#pragma unroll
            for (int e = 0; e < Sh::E; e++) x[e] = ds.d(2, j, Sh::LOG_N, last_pos<Sh>(m, tid, e), pc);
        } else {
            if (j > 0) ntt_barrier<Sh>();
            const u64 *src = a.c2 + ((size_t)c * n + j) * Sh::N;
            auto st = [&](u32, u64) {};
            // The transform takes any input below 8t + 2^32 congruent to the
            // digit: when q_j <= 8t the digit c2_j < q_j goes in as it is.
            if (a.ctx.pc[j].p <= (pc.four_p << 1)) {
                auto ld = [&](u32 P) -> u64 { return __ldg(reinterpret_cast<const unsigned long long *>(src + P)); };
                ntt_fwd_block<Sh, false>(smem, m, 0, twf, pc, ld, st, x);
            } else {
                auto ld = [&](u32 P) -> u64 {
                    return reduce_word(__ldg(reinterpret_cast<const unsigned long long *>(src + P)), pc);
                };
                ntt_fwd_block<Sh, false>(smem, m, 0, twf, pc, ld, st, x);
            }
        }
        // multiply-accumulate with the key: lazy products in [0, 4p),
        // accumulators kept in [0, 4p)
#pragma unroll
        for (int k = 0; k < 2; k++) {
            const ulonglong2 *key = a.evk + (((size_t)j * 2 + k) * (a.ctx.n_data + 1) + tp) * Sh::N;
#pragma unroll
            for (int e = 0; e < Sh::E; e++) {
                const ulonglong2 w = __ldg(key + last_pos<Sh>(m, tid, e));
                const u64 prod = mul_shoup_lazy4_asm(x[e], w.x, w.y, pc.neg_p);
                u64 &slot = acc[(k * Sh::E + e) * Sh::T + tid];
                slot = (j == 0) ? prod : reduce_once(slot + prod, pc.four_p);
            }
        }
    }
    if (t < n) {
        const u64 P_mod_q = a.ctx.cst[3 * t + 2], P_mod_q_sh = a.ctx.cst[p_shoup_index(a.ctx, t)];
#pragma unroll
        for (int k = 0; k < 2; k++) {
            u64 *dst = a.accq + (((size_t)c * 2 + k) * n + t) * Sh::N;
#pragma unroll
            for (int e = 0; e < Sh::E; e++) {
                const int P = last_pos<Sh>(m, tid, e);
                const u64 s = reduce_once(reduce_once(acc[(k * Sh::E + e) * Sh::T + tid], pc.two_p), pc.p);
                dst[P] = add_mod(s, mul_shoup(ds.d(k, t, Sh::LOG_N, (u32)P, pc), P_mod_q, P_mod_q_sh, pc.p), pc.p);
            }
        }
    } else {
        // special prime: y_k = INTT_P(acc_k) (inputs in [0, 4p)), kept in the
        // coefficient domain
#pragma unroll 1
        for (int k = 0; k < 2; k++) {
            ntt_barrier<Sh>();
#pragma unroll
            for (int e = 0; e < Sh::E; e++) x[e] = acc[(k * Sh::E + e) * Sh::T + tid];
            u64 *dst = a.plift + ((size_t)c * 2 + k) * Sh::N;
            auto st = [&](u32 P, u64 v) { dst[P] = v; };
            auto ld = [&](u32) -> u64 { return 0; };
            ntt_inv_block<Sh, true>(smem, m, 0, a.ctx.tw_inv + (size_t)tp * Sh::N, pc, ld, st, x);
        }
    }
}

// Expanded mod-up, first half: one transform per cluster,
//   X[g][t][j] = NTT_t(c2_j mod t)  for each digit j != t, target t in
//   {q_0..q_l, P}, ciphertext c = c_first + g of the group,
// left in the lazy range [0, 12t) (it only feeds Shoup products). The same
// transforms as k_ks_modup, but as independent launches of the plain
// transform's size and register budget instead of a sequence inside one
// accumulating cluster; k_ks_mac then accumulates them with the key.
// Clusters of the diagonal (j = t) exit at once: there the digit is already
// in the NTT domain.
// One transform of the expanded mod-up: X[g][t][j] = NTT_t(c2_j mod t),
// j != t, ciphertext c_first + g.
template <class Sh>
__device__ __forceinline__ void ks_expand_body(const EvalArgs &a, u32 g, u32 t, u32 j, u32 m, u32 rbase, bool valid)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 tid = threadIdx.x;
    const u32 n = a.n;
    const u32 tp = (t == n) ? a.ctx.n_data : t;
    const PrimeConst pc = a.ctx.pc[tp];
    const u64 *src = a.c2 + ((size_t)(a.c_first + g) * n + j) * Sh::N;
    u64 *dst = a.mx + (((size_t)g * (n + 1) + t) * n + j) * Sh::N;
    const ulonglong2 *twf = a.ctx.tw_fwd + (size_t)tp * Sh::N;
    u64 x[Sh::E];
    auto nost = [&](u32, u64) {};
    // any input below 8t congruent to the digit will do: when q_j <= 8t the
    // digit c2_j < q_j goes in as it is, otherwise reduce_word brings it
    // below 4t. One transform for both (the flag is uniform over the
    // item): two instances of the transform in one kernel spilled 132 bytes
    // at 64 registers, one spills 8 (measured 1.8 % off the MulLinRS batch).
    const bool reduce = a.ctx.pc[j].p > (pc.four_p << 1);
    auto ld = [&](int P) -> u64 {
        const u64 v = rd(src + P);
        return reduce ? reduce_word(v, pc) : v;
    };
    ntt_fwd_block<Sh, false>(smem, m, rbase, twf, pc, ld, nost, x);
    if (valid) store_run<Sh>(dst, x, m, tid);
}

template <int LOG_B, int LOG_C, int LOG_E, bool JOBS = false>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::MIN_CTAS)
k_ks_expand(EvalArgs a0, JobsArg<JOBS> tab)
{
    EvalArgs a = a0;
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    u32 item = blockIdx.x >> LOG_C;
    if constexpr (JOBS) item = bind_job(a, tab, JS_EXPAND, item);
    const u32 n = a.n;
    const u32 j = item % n, t = (item / n) % (n + 1), g = item / (n * (n + 1));
    if (j == t) return;   // the whole cluster: there the digit is already in the NTT domain
    ks_expand_body<Sh>(a, g, t, j, m, 0, true);
}

#ifdef HE_MISC_KERNELS
// Expanded mod-up, second half (elementwise):
//   acc_k[t] = sum_j X[g][t][j] * evk[j][k][t]   (j = t: the NTT-domain
//   digit d2_t itself), lazy products in [0, 4t), sums kept in [0, 4t);
// d_k P + acc_k, canonical, into accq for data targets (as k_ks_modup),
// acc_k left in [0, 4P) in plift for the special prime (the inverse
// transform that follows accepts that range).
// A thread takes two positions of one target for MAC_CTS ciphertexts of the
// group, so each key word it loads serves MAC_CTS products; two ciphertexts
// under a 64-register bound (four blocks of 256 per SM) measured fastest
// (one: fewer key reuses; four: too few warps to cover the loads).
constexpr u32 MAC_CTS = 2;

// One item of k_ks_mac: two positions of one target for up to MAC_CTS
// ciphertexts of the group (item q of the group's chunks x targets x pairs).
__device__ __forceinline__ void ks_mac_item(const EvalArgs &a, u32 groups, u32 q)
{
    const u32 n = a.n, N = a.ctx.N, nd1 = a.ctx.n_data + 1;
    const u32 log_n = 31 - __clz(N);
    const size_t key_j = (size_t)2 * nd1 * N, key_k = (size_t)nd1 * N;   // evk [j][k][target][N]
    const size_t mx_g = (size_t)(n + 1) * n * N;                          // mx [g][target][j][N]
    const u32 P = (q & ((N >> 1) - 1)) * 2;
    const u32 r = q >> (log_n - 1);
    const u32 t = r % (n + 1), g0 = (r / (n + 1)) * MAC_CTS;
    const u32 ng = min(MAC_CTS, groups - g0);
    const u32 tp = (t == n) ? a.ctx.n_data : t;
    const PrimeConst pc = a.ctx.pc[tp];
    const ulonglong2 *key = a.evk + (size_t)tp * N + P;                  // digit 0, k = 0
    const u64 *mx = a.mx + ((size_t)g0 * (n + 1) + t) * n * N + P;      // ciphertext g0, digit 0
    u64 acc[MAC_CTS][2][2];
    for (u32 j = 0; j < n; j++, key += key_j, mx += N) {
        ulonglong2 w[2][2];
#pragma unroll
        for (int k = 0; k < 2; k++) ld_tw2(key + k * key_k, 0, w[k][0], w[k][1]);   // positions P, P + 1
#pragma unroll
        for (u32 gi = 0; gi < MAC_CTS; gi++) {
            if (gi >= ng) break;
            ulonglong2 v;
            if (j == t)
                v = dsource(a, a.c_first + g0 + gi).d2(2, j, log_n, P, pc);
            else
                v = __ldg(reinterpret_cast<const ulonglong2 *>(mx + gi * mx_g));
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const u64 p0 = mul_shoup_lazy4_asm(v.x, w[k][0].x, w[k][0].y, pc.neg_p);
                const u64 p1 = mul_shoup_lazy4_asm(v.y, w[k][1].x, w[k][1].y, pc.neg_p);
                acc[gi][k][0] = j == 0 ? p0 : reduce_once(acc[gi][k][0] + p0, pc.four_p);
                acc[gi][k][1] = j == 0 ? p1 : reduce_once(acc[gi][k][1] + p1, pc.four_p);
            }
        }
    }
#pragma unroll
    for (u32 gi = 0; gi < MAC_CTS; gi++) {
        if (gi >= ng) break;
        const u32 c = a.c_first + g0 + gi;
        const DSource ds = dsource(a, c);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            ulonglong2 o;
            if (t < n) {
                // stored as d_k P + acc_k (see the mod-down)
                const u64 P_mod_q = a.ctx.cst[3 * t + 2], P_mod_q_sh = a.ctx.cst[p_shoup_index(a.ctx, t)];
                const u64 s0 = reduce_once(reduce_once(acc[gi][k][0], pc.two_p), pc.p);
                const u64 s1 = reduce_once(reduce_once(acc[gi][k][1], pc.two_p), pc.p);
                const ulonglong2 dv = ds.d2(k, t, log_n, P, pc);
                o.x = add_mod(s0, mul_shoup(dv.x, P_mod_q, P_mod_q_sh, pc.p), pc.p);
                o.y = add_mod(s1, mul_shoup(dv.y, P_mod_q, P_mod_q_sh, pc.p), pc.p);
                *reinterpret_cast<ulonglong2 *>(a.accq + (((size_t)c * 2 + k) * n + t) * N + P) = o;
            } else {
                o.x = acc[gi][k][0];
                o.y = acc[gi][k][1];
                *reinterpret_cast<ulonglong2 *>(a.plift + ((size_t)c * 2 + k) * N + P) = o;
            }
        }
    }
}

// Tiled form of the key multiply-accumulate for a uniform group of at
// least 8 ciphertexts: one CTA per (target t, tile of MAC_TILE positions,
// chunk of MAC_CHUNK ciphertexts). The tile's key pairs for every digit and
// component are staged in shared memory once ([2 j + k][position], 2 n
// MAC_TILE pairs) and serve every ciphertext of the chunk; each warp covers
// 4 position pairs for 8 ciphertexts (its key reads are broadcasts), each
// thread 2 positions of one ciphertext at a time, the next digit's values
// loaded while the current ones' products run. With its few registers the
// kernel runs six CTAs per SM: the per-thread form above is bound by the
// latency of its loads at four (measured: the MulLinRS batch at N = 2^14,
// 64 pairs, 1.203 -> 1.166 ms). Same products, same sums mod p: the outputs
// are those of k_ks_mac.
constexpr u32 MAC_TILE = 64, MAC_CHUNK = 32;

__global__ void __launch_bounds__(256, 6) k_ks_mac_tiled(EvalArgs a, u32 groups)
{
    extern __shared__ __align__(16) ulonglong2 key_tile[];   // [2 n][MAC_TILE]
    const u32 n = a.n, N = a.ctx.N, nd1 = a.ctx.n_data + 1;
    const u32 tiles = N / MAC_TILE, chunks = (groups + MAC_CHUNK - 1) / MAC_CHUNK;
    const u32 b = blockIdx.x;
    const u32 chunk = b % chunks, tile = (b / chunks) % tiles, t = b / (chunks * tiles);
    const u32 tp = (t == n) ? a.ctx.n_data : t;
    const PrimeConst pc = a.ctx.pc[tp];
    const u32 P0 = tile * MAC_TILE;
    for (u32 i = threadIdx.x; i < n * 2 * MAC_TILE; i += blockDim.x) {
        const u32 row = i / MAC_TILE, col = i % MAC_TILE;   // row 2 j + k: evk [j][k][target][N]
        key_tile[i] = __ldg(a.evk + ((size_t)row * nd1 + tp) * N + P0 + col);
    }
    __syncthreads();
    const u32 lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const u32 pp = warp * 4 + (lane & 3);
    const u32 P = P0 + 2 * pp;
    const u32 log_n = 31 - __clz(N);
    const u32 gend = min(groups, (chunk + 1) * MAC_CHUNK);
    for (u32 g = chunk * MAC_CHUNK + (lane >> 2); g < gend; g += 8) {
        const u64 *mxp = a.mx + ((size_t)g * (n + 1) + t) * n * N + P;   // mx [g][target][j][N]
        auto load_v = [&](u32 j) -> ulonglong2 {
            if (j == t) return dsource(a, a.c_first + g).d2(2, j, log_n, P, pc);
            return __ldg(reinterpret_cast<const ulonglong2 *>(mxp + (size_t)j * N));
        };
        u64 acc[2][2];
        ulonglong2 vn = load_v(0);
        for (u32 j = 0; j < n; j++) {
            const ulonglong2 v = vn;
            if (j + 1 < n) vn = load_v(j + 1);
#pragma unroll
            for (int k = 0; k < 2; k++) {
                const ulonglong2 w0 = key_tile[(2 * j + k) * MAC_TILE + 2 * pp];
                const ulonglong2 w1 = key_tile[(2 * j + k) * MAC_TILE + 2 * pp + 1];
                const u64 p0 = mul_shoup_lazy4_asm(v.x, w0.x, w0.y, pc.neg_p);
                const u64 p1 = mul_shoup_lazy4_asm(v.y, w1.x, w1.y, pc.neg_p);
                acc[k][0] = j == 0 ? p0 : reduce_once(acc[k][0] + p0, pc.four_p);
                acc[k][1] = j == 0 ? p1 : reduce_once(acc[k][1] + p1, pc.four_p);
            }
        }
        const u32 c = a.c_first + g;
        const DSource ds = dsource(a, c);
#pragma unroll
        for (int k = 0; k < 2; k++) {
            ulonglong2 o;
            if (t < n) {
                // stored as d_k P + acc_k (see the mod-down)
                const u64 P_mod_q = a.ctx.cst[3 * t + 2], P_mod_q_sh = a.ctx.cst[p_shoup_index(a.ctx, t)];
                const u64 s0 = reduce_once(reduce_once(acc[k][0], pc.two_p), pc.p);
                const u64 s1 = reduce_once(reduce_once(acc[k][1], pc.two_p), pc.p);
                const ulonglong2 dv = ds.d2(k, t, log_n, P, pc);
                o.x = add_mod(s0, mul_shoup(dv.x, P_mod_q, P_mod_q_sh, pc.p), pc.p);
                o.y = add_mod(s1, mul_shoup(dv.y, P_mod_q, P_mod_q_sh, pc.p), pc.p);
                *reinterpret_cast<ulonglong2 *>(a.accq + (((size_t)c * 2 + k) * n + t) * N + P) = o;
            } else {
                o.x = acc[k][0];
                o.y = acc[k][1];
                *reinterpret_cast<ulonglong2 *>(a.plift + ((size_t)c * 2 + k) * N + P) = o;
            }
        }
    }
}

// Items: for a uniform group, (groups / MAC_CTS rounded up) x (n + 1)
// targets x N / 2 position pairs; for a job table, those of every job back
// to back (each job one group of all its ciphertexts). `total` is below 2^32
// for every accepted size (64 ciphertexts per group, 33 targets, 2^15 pairs).
template <bool JOBS = false>
__global__ void __launch_bounds__(256, 4) k_ks_mac(EvalArgs a0, u32 groups, u32 total, JobsArg<JOBS> tab)
{
    for (u32 q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        if constexpr (JOBS) {
            EvalArgs a = a0;
            const u32 local = bind_job(a, tab, JS_MAC, q);
            ks_mac_item(a, a.count, local);
        } else {
            ks_mac_item(a0, groups, q);
        }
    }
}
#endif  // HE_MISC_KERNELS

// Relin mod-down (no rescale): out[c][k][i] = d_k[i] + (acc - NTT(r)) P^-1.
template <int LOG_B, int LOG_C, int LOG_E>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::EVAL_MIN_CTAS)
k_ks_moddown(EvalArgs a)
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(16) u64 smem[];
    const u32 tid = threadIdx.x;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 item = blockIdx.x >> LOG_C;
    const u32 n = a.n;
    const u32 c = item / (2 * n), k = (item / n) % 2, i = item % n;
    const PrimeConst pc = a.ctx.pc[i];
    const PrimeConst pP = a.ctx.pc[a.ctx.n_data];
    const u64 *cst = a.ctx.cst + 3 * i;         // P^-1, Shoup, P mod q_i
    const u64 half_P = (pP.p - 1) / 2;
    const u64 *y = a.plift + ((size_t)c * 2 + k) * Sh::N;
    u64 x[Sh::E];
    auto ld = [&](u32 P) -> u64 { return centred_mod(rd(y + P), half_P, cst[2], pc); };
    auto st = [&](u32, u64) {};
    ntt_fwd_block<Sh, false>(smem, m, 0, a.ctx.tw_fwd + (size_t)i * Sh::N, pc, ld, st, x);
    const u64 *accp = a.accq + (((size_t)c * 2 + k) * n + i) * Sh::N;
    u64 *out = a.out + (((size_t)c * 2 + k) * n + i) * Sh::N;
    sub_scale_run<Sh>(x, accp, cst[0], cst[1], pc, m, tid);   // acc holds d P
    store_run<Sh>(out, x, m, tid);
}

// RS, first half: y_k = INTT_{q_l}(c_k[q_l]) -> lift2 (coefficient domain).
template <int LOG_B, int LOG_C, int LOG_E>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::EVAL_MIN_CTAS)
k_rs_lift(EvalArgs a)
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(16) u64 smem[];
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 item = blockIdx.x >> LOG_C;
    const u32 n = a.n, l = n - 1;
    const u32 c = item / 2, k = item % 2;
    const PrimeConst pc = a.ctx.pc[l];
    const u64 *src = a.ct2 + (((size_t)c * 2 + k) * n + l) * Sh::N;
    u64 *dst = a.lift2 + ((size_t)c * 2 + k) * Sh::N;
    u64 x[Sh::E];
    auto ld = [&](u32 P) -> u64 { return rd(src + P); };
    auto st = [&](u32 P, u64 v) { dst[P] = v; };
    ntt_inv_block<Sh, false>(smem, m, 0, a.ctx.tw_inv + (size_t)l * Sh::N, pc, ld, st, x);
}

// RS, second half: out[c][k][i] = (c_k[q_i] - NTT(r mod q_i)) q_l^-1, i < l.
template <int LOG_B, int LOG_C, int LOG_E>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::EVAL_MIN_CTAS)
k_rs(EvalArgs a)
{
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    extern __shared__ __align__(16) u64 smem[];
    const u32 tid = threadIdx.x;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    const u32 item = blockIdx.x >> LOG_C;
    const u32 n = a.n, l = n - 1;
    const u32 c = item / (2 * l), k = (item / l) % 2, i = item % l;
    const PrimeConst pc = a.ctx.pc[i];
    const u64 *cst = a.ctx.cst + 3 * a.ctx.n_data + 3 * ((size_t)l * a.ctx.n_data + i);
    const u64 half_l = (a.ctx.pc[l].p - 1) / 2;
    const u64 *y = a.lift2 + ((size_t)c * 2 + k) * Sh::N;
    u64 x[Sh::E];
    auto ld = [&](u32 P) -> u64 { return centred_mod(rd(y + P), half_l, cst[2], pc); };
    auto st = [&](u32, u64) {};
    ntt_fwd_block<Sh, false>(smem, m, 0, a.ctx.tw_fwd + (size_t)i * Sh::N, pc, ld, st, x);
    const u64 *src = a.ct2 + (((size_t)c * 2 + k) * n + i) * Sh::N;
    u64 *out = a.out + (((size_t)c * 2 + k) * l + i) * Sh::N;
    sub_scale_run<Sh>(x, src, cst[0], cst[1], pc, m, tid);
    store_run<Sh>(out, x, m, tid);
}

// MulLinRS, limb q_l: relin output c_k[q_l] = d_k[l] + (acc - NTT(r)) P^-1,
// then straight into INTT_{q_l} (values stay in registers) -> lift2;
// item = 2 c + k.
template <class Sh>
__device__ __forceinline__ void mrr_last_body(const EvalArgs &a, u32 item, u32 m, u32 rbase, bool valid)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 tid = threadIdx.x;
    const u32 n = a.n, l = n - 1;
    const u32 c = item / 2, k = item % 2;
    const PrimeConst pc = a.ctx.pc[l];
    const PrimeConst pP = a.ctx.pc[a.ctx.n_data];
    const u64 *cst = a.ctx.cst + 3 * l;
    const u64 half_P = (pP.p - 1) / 2;
    const u64 *y = a.plift + ((size_t)c * 2 + k) * Sh::N;
    u64 x[Sh::E];
    auto ld = [&](u32 P) -> u64 { return centred_mod(rd(y + P), half_P, cst[2], pc); };
    auto nost = [&](u32, u64) {};
    ntt_fwd_block<Sh, false>(smem, m, rbase, a.ctx.tw_fwd + (size_t)l * Sh::N, pc, ld, nost, x);
    const u64 *accp = a.accq + (((size_t)c * 2 + k) * n + l) * Sh::N;
    sub_scale_run<Sh>(x, accp, cst[0], cst[1], pc, m, tid);   // acc holds d P
    u64 *dst = a.lift2 + ((size_t)c * 2 + k) * Sh::N;
    auto st = [&](u32 P, u64 v) {
        if (valid) dst[P] = v;
    };
    auto nold = [&](u32) -> u64 { return 0; };
    ntt_inv_block<Sh, true>(smem, m, rbase, a.ctx.tw_inv + (size_t)l * Sh::N, pc, nold, st, x);
}

template <int LOG_B, int LOG_C, int LOG_E, bool JOBS = false>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::EVAL_MIN_CTAS)
k_mrr_last(EvalArgs a0, JobsArg<JOBS> tab)
{
    EvalArgs a = a0;
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    u32 item = blockIdx.x >> LOG_C;
    if constexpr (JOBS) item = bind_job(a, tab, JS_LAST, item);
    mrr_last_body<Sh>(a, item, m, 0, true);
}

// MulLinRS, limbs i < l: mod-down by P, then rescale by q_l, as two launches
// of one transform each (plain transform size and register budget; one
// fused kernel holding the first result across the second transform needs
// twice the registers):
//   k_mrr_rest_z:   z_k[i] = d_k[i] + (acc_k[i] - NTT_i([y_k]_P)) P^-1
//                          = (stored acc - NTT_i([y_k]_P)) P^-1 (the mod-up
//                   stores d_k P + acc_k), written over the accumulator (each
//                   thread rewrites only the positions it read);
//   k_mrr_rest_out: out[c][k][i] = (z_k[i] - NTT_i([y2_k]_{q_l})) q_l^-1.
// Both transforms are left lazy (their outputs only enter Shoup products).
// item = 2 l c + l k + i (ciphertext c, component k, limb i < l).
template <class Sh>
__device__ __forceinline__ void mrr_rest_z_body(const EvalArgs &a, u32 item, u32 m, u32 rbase, bool valid)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 tid = threadIdx.x;
    const u32 n = a.n, l = n - 1;
    const u32 c = item / (2 * l), k = (item / l) % 2, i = item % l;
    const PrimeConst pc = a.ctx.pc[i];
    const u64 *cP = a.ctx.cst + 3 * i;
    const u64 half_P = (a.ctx.pc[a.ctx.n_data].p - 1) / 2;
    const u64 P_mod_q = cP[2];
    const u64 *y = a.plift + ((size_t)c * 2 + k) * Sh::N;
    u64 x[Sh::E];
    auto nost = [&](u32, u64) {};
    auto ld = [&](int P) -> u64 { return centred_mod(rd(y + P), half_P, P_mod_q, pc); };
    ntt_fwd_block<Sh, false>(smem, m, rbase, a.ctx.tw_fwd + (size_t)i * Sh::N, pc, ld, nost, x);
    u64 *accp = a.accq + (((size_t)c * 2 + k) * n + i) * Sh::N;
    sub_scale_run<Sh>(x, accp, cP[0], cP[1], pc, m, tid);
    if (valid) store_run<Sh>(accp, x, m, tid);
}

template <class Sh>
__device__ __forceinline__ void mrr_rest_out_body(const EvalArgs &a, u32 item, u32 m, u32 rbase, bool valid)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 tid = threadIdx.x;
    const u32 n = a.n, l = n - 1;
    const u32 c = item / (2 * l), k = (item / l) % 2, i = item % l;
    const PrimeConst pc = a.ctx.pc[i];
    const u64 *cl = a.ctx.cst + 3 * a.ctx.n_data + 3 * ((size_t)l * a.ctx.n_data + i);
    const u64 half_l = (a.ctx.pc[l].p - 1) / 2;
    const u64 ql_mod_q = cl[2];
    const u64 *y2 = a.lift2 + ((size_t)c * 2 + k) * Sh::N;
    u64 x[Sh::E];
    auto nost = [&](u32, u64) {};
    auto ld = [&](int P) -> u64 { return centred_mod(rd(y2 + P), half_l, ql_mod_q, pc); };
    ntt_fwd_block<Sh, false>(smem, m, rbase, a.ctx.tw_fwd + (size_t)i * Sh::N, pc, ld, nost, x);
    const u64 *zp = a.accq + (((size_t)c * 2 + k) * n + i) * Sh::N;
    u64 *out = a.out + (((size_t)c * 2 + k) * l + i) * Sh::N;
    sub_scale_run<Sh>(x, zp, cl[0], cl[1], pc, m, tid);
    if (valid) store_run<Sh>(out, x, m, tid);
}

// Inverse transform of one special-prime accumulator row of plift in place
// (row = 2 c + k; inputs in [0, 4P), the key multiply-accumulate's range).
// Every load precedes the cluster barrier before the cross-CTA stages (or,
// in one CTA, the barrier of the first round exchange) and every store
// follows it, so the rows can be transformed in place.
template <class Sh>
__device__ __forceinline__ void plift_intt_body(const EvalArgs &a, u32 row, u32 m, u32 rbase, bool valid)
{
    extern __shared__ __align__(16) u64 smem[];
    const u32 tp = a.ctx.n_data;
    u64 *y = a.plift + (size_t)row * Sh::N;
    u64 x[Sh::E];
    auto ld = [&](u32 P) -> u64 { return rd(y + P); };
    auto st = [&](u32 P, u64 v) {
        if (valid) y[P] = v;
    };
    ntt_inv_block<Sh, false>(smem, m, rbase, a.ctx.tw_inv + (size_t)tp * Sh::N, a.ctx.pc[tp], ld, st, x);
}

template <int LOG_B, int LOG_C, int LOG_E, bool JOBS = false>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::MIN_CTAS)
k_mrr_rest_z(EvalArgs a0, JobsArg<JOBS> tab)
{
    EvalArgs a = a0;
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    u32 item = blockIdx.x >> LOG_C;
    if constexpr (JOBS) item = bind_job(a, tab, JS_REST, item);
    mrr_rest_z_body<Sh>(a, item, m, 0, true);
}

template <int LOG_B, int LOG_C, int LOG_E, bool JOBS = false>
__global__ void __launch_bounds__(NttShape<LOG_B, LOG_C, LOG_E>::T, NttShape<LOG_B, LOG_C, LOG_E>::MIN_CTAS)
k_mrr_rest_out(EvalArgs a0, JobsArg<JOBS> tab)
{
    EvalArgs a = a0;
    using Sh = NttShape<LOG_B, LOG_C, LOG_E>;
    const u32 m = (LOG_C > 0) ? cluster_ctarank() : 0u;
    u32 item = blockIdx.x >> LOG_C;
    if constexpr (JOBS) item = bind_job(a, tab, JS_REST, item);
    mrr_rest_out_body<Sh>(a, item, m, 0, true);
}

}  // namespace he
