// CUDA kernels of libfem for sm_103a: one explicit EBE enthalpy step
// (Eq. 14 in the enthalpy form of Eq. 5, element sums of Eqs. 15-22), the
// interface load of Eq. 8 and the flat (atomic, coloured) variants.  The
// state I/O and energy kernels are in fem_io.cu.
//
// Block variant (the hot path):
//   k_block_step      one CTA per element block.  Pass 1 turns the block's
//                     nodal enthalpies into temperatures T(E) (Eqs. 5, 11)
//                     and writes each node's T into the shared-memory slots
//                     of its element corners; pass 2 forms r = -K^e T^e for
//                     every element from the six stored conductances
//                     (Eq. 18: only K^e is stored) and the Robin face terms
//                     (Eq. 4); pass 3 sums each node's slots in a fixed
//                     order (no atomics) and updates interior nodes
//                     E += dt R, or writes the partial sum of a node shared
//                     with other blocks (the exchange of calculated values,
//                     Eqs. 19-22).
//   k_shared_update   sums the partials of every shared node in a fixed
//                     order and updates it.
// The step accumulates, in FP64 per CTA, the heat that entered through the
// Robin faces; the state functions sum E and latent heat still to release
// are FP64 reductions of the state taken on demand (fem_io.cu).
#include <cuda_runtime.h>

#include <cstdint>

#include "fem_internal.h"
#include "fem_device.cuh"

#include "fem_state.cuh"

namespace fem {

namespace {

// ---------------------------------------------------------------------------
// Block variant
// ---------------------------------------------------------------------------

// A bulk copy did not complete in time: flag it and give the copies a
// bounded second chance to land before the CTA releases its shared memory
// (every thread of the CTA calls this, then returns).
__device__ __forceinline__ void give_up(int *err, uint32_t bar_s, uint32_t bar_w, uint32_t bar_n)
{
    if (threadIdx.x == 0) {
        atomicExch(err, kErrWaitTimeout);
        mbar_wait(bar_n, 0);
        mbar_wait(bar_s, 0);
        mbar_wait(bar_w, 0);
    }
    __syncthreads();
}

// k(T) of material m: its table of n points (T_j ascending), linear between
// points, constant beyond the ends (the reading of Eq. 9's K(T)).
template <typename real>
__device__ __forceinline__ real conductivity_of(const real *kt_T, const real *kt_k,
                                                const int32_t *kt_n, int m, real T)
{
    const int n = __ldg(kt_n + m);
    const real *Tj = kt_T + m * kKtMax, *kj = kt_k + m * kKtMax;
    if (T <= __ldg(Tj)) return __ldg(kj);
    if (T >= __ldg(Tj + n - 1)) return __ldg(kj + n - 1);
    int j = 0;
    while (T > __ldg(Tj + j + 1)) j++;
    const real T0 = __ldg(Tj + j), k0 = __ldg(kj + j);
    return k0 + (__ldg(kj + j + 1) - k0) * (T - T0) / (__ldg(Tj + j + 1) - T0);
}

// Apparent specific heat of one element by Lemmon's method (Eq. 7): the
// ratio of the gradient magnitudes of H(T) = c T + L f_l(T) and of T over the
// element.  With the six conductances (K^e has zero row sums), |grad x|^2 is
// proportional to sum_{a<b} w_ab (x_a - x_b)^2, so the common factor cancels;
// where T is uniform over the element (every difference below a
// micro-kelvin) dH/dT at the mean temperature is used.
template <typename real>
__device__ __forceinline__ real apparent_cp(const BlockArgs<real> &a, int m, real T0, real T1, real T2,
                                            real T3, real w01, real w02, real w03, real w12,
                                            real w13, real w23)
{
    const real c = __ldg(a.lm_c + m), L = __ldg(a.lm_L + m);
    if (!(L > real(0))) return c;
    const real Ts = __ldg(a.lm_Ts + m), Tl = __ldg(a.lm_Tl + m), inv = real(1) / (Tl - Ts);
    auto H = [&](real T) {
        const real f = T <= Ts ? real(0) : (T >= Tl ? real(1) : (T - Ts) * inv);
        return c * T + L * f;
    };
    const real H0 = H(T0), H1 = H(T1), H2 = H(T2), H3 = H(T3);
    const real num = w01 * (H0 - H1) * (H0 - H1) + w02 * (H0 - H2) * (H0 - H2) +
                     w03 * (H0 - H3) * (H0 - H3) + w12 * (H1 - H2) * (H1 - H2) +
                     w13 * (H1 - H3) * (H1 - H3) + w23 * (H2 - H3) * (H2 - H3);
    const real den = w01 * (T0 - T1) * (T0 - T1) + w02 * (T0 - T2) * (T0 - T2) +
                     w03 * (T0 - T3) * (T0 - T3) + w12 * (T1 - T2) * (T1 - T2) +
                     w13 * (T1 - T3) * (T1 - T3) + w23 * (T2 - T3) * (T2 - T3);
    const real wsum = ((w01 + w02) + (w03 + w12)) + (w13 + w23);
    if (den > real(1e-12) * wsum) return sqrt(num / den);
    const real Tm = (T0 + T1 + T2 + T3) * real(0.25);
    return (Tm >= Ts && Tm < Tl) ? c + L * inv : c;
}

// Capacity behind a slot of the block's slot array: element-corner slots
// (below 4 ne_pad) name element slot - corner * ne_pad, whose capacity pass
// 2 left at sw[element]; face and padding slots carry none.
template <typename real>
__device__ __forceinline__ real slot_capacity(const real *sw, uint32_t v, int ne_pad)
{
    const int sl = (int)v;
    if (sl >= 4 * ne_pad) return real(0);
    const int c = (sl >= ne_pad) + (sl >= 2 * ne_pad) + (sl >= 3 * ne_pad);
    return sw[sl - c * ne_pad];
}

// The 32-lane schedule group that warp `warp` handles in its j-th slot (-1:
// none), for NW warps and ngrp groups.  Groups come longest first (nodes are
// ordered by slot count); when there are between NW and 2 NW of them the
// longest get a warp each and the rest are paired long with short on the
// remaining warps, so that no warp's work exceeds the longest group's.
template <int NW, int MAXJ>
__device__ __forceinline__ int block_group(int warp, int j, int ngrp)
{
    if (ngrp <= NW) return j == 0 && warp < ngrp ? warp : -1;
    if (MAXJ >= 2 && ngrp <= 2 * NW) {
        const int extra = ngrp - NW;
        if (warp < NW - extra) return j == 0 ? warp : -1;
        const int i = warp - (NW - extra);
        return j == 0 ? NW - extra + i : (j == 1 ? ngrp - 1 - i : -1);
    }
    const int g = warp + j * NW;
    return g < ngrp ? g : -1;
}

// Element product of one tet: r_a = sum_b w_ab (T_b - T_a), w_ab = -K^e_ab
// (the row of -K^e T^e; K^e symmetric with zero row sums, Eq. 9).
template <typename real>
__device__ __forceinline__ void tet_products(real w01, real w02, real w03, real w12, real w13,
                                             real w23, real T0, real T1, real T2, real T3,
                                             real &r0, real &r1, real &r2, real &r3)
{
    const real p01 = w01 * (T1 - T0), p02 = w02 * (T2 - T0), p03 = w03 * (T3 - T0);
    const real p12 = w12 * (T2 - T1), p13 = w13 * (T3 - T1), p23 = w23 * (T3 - T2);
    r0 = p01 + p02 + p03;
    r1 = (p12 + p13) - p01;
    r2 = p23 - (p02 + p12);
    r3 = -(p03 + p13 + p23);
}

template <typename real>
struct Vec2Of;
template <>
struct Vec2Of<float> {
    using type = float2;
};
template <>
struct Vec2Of<double> {
    using type = double2;
};

template <typename real>
struct Vec4Of;
template <>
struct Vec4Of<float> {
    using type = float4;   // four elements per 16-byte access
    static constexpr int n = 4;
};
template <>
struct Vec4Of<double> {
    using type = double2;  // two elements per 16-byte access
    static constexpr int n = 2;
};

// 16-byte vector of `real` accessed by lane index
__device__ __forceinline__ float &vat(float4 &v, int i) { return (&v.x)[i]; }
__device__ __forceinline__ double &vat(double2 &v, int i) { return (&v.x)[i]; }

// One CTA per element block b, NT threads.  The block's local node data
// (stride b*ls), schedule chunk (stride b*chunk_words) and six conductance
// rows (stride 6*b*nes) all sit at fixed strides, so thread 0 bulk-copies
// them into shared memory at kernel start from blockIdx alone.
// A warp owns the 32-lane schedule groups block_group() gives it (group g
// covers local nodes 32 g + lane); thread t owns element quad(s) t, t+NT, ...
// WG: the conductances are not staged in shared memory; pass 2 reads them
// from global memory, brought into L2 by a bulk prefetch at the start of
// the CTA.  A 1,792-tet FP32 block then needs ~56 KB, and four CTAs of 256
// threads (64 registers) share an SM.
template <typename real, int NT, bool KT, bool LM, bool WG = false>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 4 : (NT <= 512 ? 2 : 1)))
    k_block_step(const BlockArgs<real> a, const real dt)
{
    constexpr int NW = NT / 32;
    constexpr int MAXJ = kMaxLocalNodes / NT;   // local nodes per thread
    using V = typename Vec4Of<real>::type;
    using V2 = typename Vec2Of<real>::type;
    constexpr int VN = Vec4Of<real>::n;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ double qwarp[NW];   // per-warp boundary heat
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int b = a.b_first + (int)blockIdx.x;
    const int ls = a.ls, nes = a.nes;

    // shared memory: [3 barriers, block header][conductances 6 x nes]
    // [schedule chunk][slots + dummy][per local node: E, partial position,
    // phase byte]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw);
    const BlockInfo &bi = *reinterpret_cast<const BlockInfo *>(smem_raw + kSmemHdrOffset);
    real *sw = reinterpret_cast<real *>(smem_raw + kSmemBarBytes);
    uint32_t *chunk = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(sw) +
                                                    (WG ? 0 : align16(6 * (size_t)nes * sizeof(real))));
    real *sv = reinterpret_cast<real *>(reinterpret_cast<unsigned char *>(chunk) +
                                        align16((size_t)a.chunk_words * 4));
    real *sE = sv + a.max_slots;                                  // [ls]
    int32_t *sPos = reinterpret_cast<int32_t *>(sE + ls);         // [ls]
    uint8_t *sPh = reinterpret_cast<uint8_t *>(sPos + ls);        // [ls]
    const uint32_t bar_s = smem_addr(bar), bar_w = smem_addr(bar + 1), bar_n = smem_addr(bar + 2);
    const size_t lb = (size_t)b * ls;

    // bulk copies: the local node data first (fixed stride, needed first;
    // (C, Lc) goes to the slot area, free until pass 1), then the schedule
    // chunk and the six conductance rows named by the block header
    if (threadIdx.x == 0) {
        mbar_init(bar_s, 1);
        mbar_init(bar_w, 1);
        mbar_init(bar_n, 1);
        mbar_fence_init();
        const uint32_t eb = (uint32_t)(ls * sizeof(real));
        // E, (C, Lc), phase, position, and the block header
        mbar_arrive_expect_tx(bar_n, 3u * eb + 5u * (uint32_t)ls + (uint32_t)sizeof(BlockInfo));
        bulk_load(smem_addr(smem_raw + kSmemHdrOffset), a.blocks + b, (uint32_t)sizeof(BlockInfo), bar_n);
        bulk_load(smem_addr(sE), a.Eloc + lb, eb, bar_n);
        bulk_load(smem_addr(sv), a.CLloc + 2 * lb, 2 * eb, bar_n);
        bulk_load(smem_addr(sPh), a.phloc + lb, (uint32_t)ls, bar_n);
        bulk_load(smem_addr(sPos), a.posloc + lb, (uint32_t)ls * 4u, bar_n);
        // the schedule chunk (fixed stride) and the six conductance rows:
        // every copy is in flight before the block header is read
        const uint32_t bytes = (uint32_t)a.chunk_words * 4u;
        mbar_arrive_expect_tx(bar_s, bytes);
        bulk_load(smem_addr(chunk), a.sched + (size_t)b * a.chunk_words, bytes, bar_s);
        const uint32_t wbytes = (uint32_t)(6 * (size_t)nes * sizeof(real));
        if (WG) {   // bar_w completes at once (the fault hook leaves it
                    // waiting for bytes that never come); rows go to L2 only
            mbar_arrive_expect_tx(bar_w, a.fault_skip_weights ? wbytes : 0u);
            bulk_prefetch_l2(a.w + 6 * (size_t)b * nes, wbytes);
        } else {
            mbar_arrive_expect_tx(bar_w, wbytes);
            if (!a.fault_skip_weights) bulk_load(smem_addr(sw), a.w + 6 * (size_t)b * nes, wbytes, bar_w);
        }
    }
    // this block's time step (a batch gives every instance its own; the
    // load's latency is hidden behind the passes)
    const real dtb = a.blk_dt ? a.blk_dt[b] : dt;

    // thread 0 initialised the mbarriers before it waits on bar_n; the other
    // threads touch them only after the vote below, which orders the two
    int failed = 0;
    if (threadIdx.x == 0) failed = !mbar_wait(bar_n, 0);
    if (__syncthreads_or(failed)) {
        give_up(a.err, bar_s, bar_w, bar_n);
        return;
    }
    mbar_try_wait(bar_n, 0);
    // the block header is in shared memory from here on
    const int nloc = bi.nint + bi.nsh;
    const int ne_pad = bi.ne_pad, nf_pad = bi.nf_pad;
    const int dummy = 4 * ne_pad + 3 * nf_pad;
    const int hdr = (bi.ngrp + 4) & ~3;   // header words: ngrp+1 group offsets, padded to 16 B
    // k(T): the materials of this thread's first element quad, loaded now
    // and used in pass 2
    uint32_t mat_q = 0;
    V rv_q{};   // apparent capacity: rho V / 4 of the quad's elements
    if ((KT || LM) && (int)threadIdx.x * VN < bi.ne) {
        const uint8_t *pm = a.emat + (size_t)b * nes + threadIdx.x * VN;
        mat_q = VN == 4 ? *reinterpret_cast<const uint32_t *>(pm)
                        : (uint32_t)*reinterpret_cast<const uint16_t *>(pm);
        if (LM) rv_q = *reinterpret_cast<const V *>(a.rv + (size_t)b * nes + threadIdx.x * VN);
    }
    // this thread's first face; thread 0: the block's boundary heat so far
    // (loads whose latency the passes below hide)
    real fa0 = real(0), fg0 = real(0);
    if ((int)threadIdx.x < bi.nf) {
        fa0 = __ldg(a.fa + bi.f0 + threadIdx.x);
        fg0 = __ldg(a.fg + bi.f0 + threadIdx.x);
    }
    double qprev = 0.0;
    if (threadIdx.x == 0 && bi.nf > 0) qprev = a.qcum[b];

    // local nodes: enthalpy -> temperature (Eqs. 5, 11); padding entries
    // hold 1/C = 1, Lc = 0 and give a harmless T
    real Tl[MAXJ];
#pragma unroll
    for (int j = 0; j < MAXJ; j++) {
        const int g = block_group<NW, MAXJ>(warp, j, bi.ngrp);
        const int l = 32 * g + lane;
        Tl[j] = real(0);
        if (g >= 0 && l < ls) {
            if (LM) {   // the state is T
                Tl[j] = sE[l];
            } else {
                const V2 cl = reinterpret_cast<const V2 *>(sv)[l];   // (1/C, Lc)
                Tl[j] = temperature_of_rc(sE[l], cl.x, cl.y, sPh[l], a.ranges);
            }
        }
    }
    // the vote below is also the barrier that ends the reads of (1/C, Lc)
    // from the slot area before pass 1 overwrites it
    if (threadIdx.x == 0) failed = !mbar_wait(bar_s, 0);
    if (__syncthreads_or(failed)) {
        give_up(a.err, bar_s, bar_w, bar_n);
        return;
    }
    mbar_try_wait(bar_s, 0);
    const uint32_t *pairs = chunk + hdr;   // pair p, lane l at pairs[p*32 + l]

    // pass 1: T of every local node into the slots of its element corners
    // (padding entries all name the dummy slot)
#pragma unroll
    for (int j = 0; j < MAXJ; j++) {
        const int g = block_group<NW, MAXJ>(warp, j, bi.ngrp);
        if (g >= 0) {
            const int p0 = (int)chunk[g], p1 = (int)chunk[g + 1];
            const real T = Tl[j];
#pragma unroll 4
            for (int pr = p0; pr < p1; ++pr) {
                const uint32_t v = pairs[pr * 32 + lane];
                if (FEM_IN(v & 0xFFFFu, a.max_slots, a.err)) sv[v & 0xFFFFu] = T;
                if (FEM_IN(v >> 16, a.max_slots, a.err)) sv[v >> 16] = T;
            }
        }
    }

    if (threadIdx.x == 0) failed = !mbar_wait(bar_w, 0);
    if (__syncthreads_or(failed)) {
        give_up(a.err, bar_s, bar_w, bar_n);
        return;
    }
    mbar_try_wait(bar_w, 0);

    // pass 2: element products, VN elements per 16-byte access
    for (int qd = threadIdx.x; qd * VN < bi.ne; qd += NT) {
        const int e = qd * VN;
        if (!FEM_IN(e + VN - 1, nes, a.err) || !FEM_IN(3 * ne_pad + e + VN - 1, a.max_slots, a.err)) break;
        V wq[6];
#pragma unroll
        for (int k = 0; k < 6; k++)
            wq[k] = WG ? __ldg(reinterpret_cast<const V *>(a.w + (6 * (size_t)b + k) * nes + e))
                       : *reinterpret_cast<const V *>(sw + k * nes + e);
        V T0 = *reinterpret_cast<const V *>(sv + e);
        V T1 = *reinterpret_cast<const V *>(sv + ne_pad + e);
        V T2 = *reinterpret_cast<const V *>(sv + 2 * ne_pad + e);
        V T3 = *reinterpret_cast<const V *>(sv + 3 * ne_pad + e);
        uint32_t mq = mat_q;
        V rvq = rv_q;
        if ((KT || LM) && qd != (int)threadIdx.x) {
            const uint8_t *pm = a.emat + (size_t)b * nes + e;
            mq = VN == 4 ? *reinterpret_cast<const uint32_t *>(pm)
                         : (uint32_t)*reinterpret_cast<const uint16_t *>(pm);
            if (LM) rvq = *reinterpret_cast<const V *>(a.rv + (size_t)b * nes + e);
        }
        V capq{};
        if (LM) {   // apparent specific heat (Eq. 7) x rho V / 4 per element
#pragma unroll
            for (int i = 0; i < VN; i++) {
                const int mt = (int)((mq >> (8 * i)) & 0xFFu);
                vat(capq, i) = vat(rvq, i) * apparent_cp(a, mt, vat(T0, i), vat(T1, i), vat(T2, i),
                                                         vat(T3, i), vat(wq[0], i), vat(wq[1], i),
                                                         vat(wq[2], i), vat(wq[3], i), vat(wq[4], i),
                                                         vat(wq[5], i));
            }
        }
        if (KT) {   // K^e(T) = k(mean element temperature) x the k = 1 weights
#pragma unroll
            for (int i = 0; i < VN; i++) {
                const real Tm = (vat(T0, i) + vat(T1, i) + vat(T2, i) + vat(T3, i)) * real(0.25);
                const real kk = conductivity_of(a.kt_T, a.kt_k, a.kt_n, (int)((mq >> (8 * i)) & 0xFFu), Tm);
#pragma unroll
                for (int k = 0; k < 6; k++) vat(wq[k], i) *= kk;
            }
        }
#pragma unroll
        for (int i = 0; i < VN; i++)
            tet_products(vat(wq[0], i), vat(wq[1], i), vat(wq[2], i), vat(wq[3], i), vat(wq[4], i),
                         vat(wq[5], i), vat(T0, i), vat(T1, i), vat(T2, i), vat(T3, i), vat(T0, i),
                         vat(T1, i), vat(T2, i), vat(T3, i));
        *reinterpret_cast<V *>(sv + e) = T0;
        *reinterpret_cast<V *>(sv + ne_pad + e) = T1;
        *reinterpret_cast<V *>(sv + 2 * ne_pad + e) = T2;
        *reinterpret_cast<V *>(sv + 3 * ne_pad + e) = T3;
        // the element capacities go over the first conductance row, which
        // only this thread reads (its own quad, already in registers)
        if (LM) *reinterpret_cast<V *>(sw + e) = capq;
    }
    if (threadIdx.x == 0) sv[dummy] = real(0);   // padding adds nothing in pass 3
    // Robin faces (Eq. 4): r_c = A/3 (h T_inf - q) - h A/12 (T_c + T_0 + T_1 + T_2)
    real qin = real(0);   // heat entering through this thread's faces
    for (int f = threadIdx.x; f < bi.nf; f += NT) {
        real *s0 = sv + 4 * ne_pad + f;
        const real T0 = s0[0], T1 = s0[nf_pad], T2 = s0[2 * nf_pad];
        const bool first = f == (int)threadIdx.x;
        const real ha = first ? fa0 : __ldg(a.fa + bi.f0 + f);
        const real hg = first ? fg0 : __ldg(a.fg + bi.f0 + f);
        const real S = T0 + T1 + T2;
        const real r0 = hg - ha * (T0 + S), r1 = hg - ha * (T1 + S), r2 = hg - ha * (T2 + S);
        s0[0] = r0;
        s0[nf_pad] = r1;
        s0[2 * nf_pad] = r2;
        qin += (r0 + r1) + r2;
    }
    if (bi.nf > 0) {   // block-uniform: per-warp partials, FP64 from there on
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) qin += __shfl_down_sync(0xffffffffu, qin, o);
        if (lane == 0) qwarp[warp] = (double)qin;
    }
    __syncthreads();

    // pass 3: fixed-order node sums; interior update or shared partial
#pragma unroll
    for (int j = 0; j < MAXJ; j++) {
        const int g = block_group<NW, MAXJ>(warp, j, bi.ngrp);
        if (g < 0) continue;
        const int l = 32 * g + lane;
        const int p0 = (int)chunk[g], p1 = (int)chunk[g + 1];
        real R = real(0), Cap = real(0);
#pragma unroll 4
        for (int pr = p0; pr < p1; ++pr) {
            const uint32_t v = pairs[pr * 32 + lane];
            if (FEM_IN(v & 0xFFFFu, a.max_slots, a.err)) R += sv[v & 0xFFFFu];
            if (FEM_IN(v >> 16, a.max_slots, a.err)) R += sv[v >> 16];
            if (LM) {   // capacity of the element behind each element-corner slot
                Cap += slot_capacity(sw, v & 0xFFFFu, ne_pad);
                Cap += slot_capacity(sw, v >> 16, ne_pad);
            }
        }
        if (l < bi.nint) {
            if (!(sPh[l] & kDirichletBit) && FEM_IN(l, ls, a.err))
                a.Eloc[lb + l] = LM ? sE[l] + dtb * R / Cap : sE[l] + dtb * R;
        } else if (l < nloc && FEM_IN(l, ls, a.err) && FEM_IN(sPos[l], a.n_copies, a.err)) {
            a.P[sPos[l]] = R;
            if (LM) a.Pc[sPos[l]] = Cap;
        }
    }
    // cumulative boundary heat of the blocks that own Robin faces (FP64)
    if (bi.nf > 0 && threadIdx.x == 0) {
        double q = 0.0;
        for (int k = 0; k < NW; k++) q += qwarp[k];
        a.qcum[b] = qprev + (double)dtb * q;
    }
}

// Shared nodes: sum the partials of every copy in a fixed order (Eq. 22),
// update E and refresh the copies' mirrors in the blocks' local arrays.
// With update == false only the mirrors are refreshed.  Each thread takes
// NPT nodes NT apart, so that their independent load chains overlap.
template <typename real, int NT, int NPT>
__global__ void __launch_bounds__(NT) k_shared_update(const BlockArgs<real> a, const real dt,
                                                      const bool update)
{
    const int64_t base = a.s_first + (int64_t)blockIdx.x * NT * NPT + threadIdx.x;
    int k0[NPT], k1[NPT];
    real E[NPT], dts[NPT];
    bool act[NPT];
#pragma unroll
    for (int j = 0; j < NPT; j++) {
        const int64_t s = base + (int64_t)j * NT;
        act[j] = s < a.s_end;
        k0[j] = k1[j] = 0;
        E[j] = dts[j] = real(0);
        if (act[j]) {
            k0[j] = __ldg(a.sh_ptr + s);
            k1[j] = __ldg(a.sh_ptr + s + 1);
            E[j] = a.Esh[s];
            if (update) {
                if (__ldg(a.ph + a.n_int + s) & kDirichletBit) act[j] = false;
                dts[j] = a.sh_dt ? a.sh_dt[s] : dt;
            }
        }
    }
    if (update) {
        real R[NPT], Cp[NPT];
#pragma unroll
        for (int j = 0; j < NPT; j++) {
            R[j] = Cp[j] = real(0);
            if (k1[j] > k0[j] && !FEM_IN(k1[j] - 1, a.n_copies, a.err)) k1[j] = k0[j];
            for (int k = k0[j]; k < k1[j]; ++k) R[j] += a.P[k];   // block order
            if (a.Pc)   // apparent capacity: T += dt R / C_app
                for (int k = k0[j]; k < k1[j]; ++k) Cp[j] += a.Pc[k];
        }
#pragma unroll
        for (int j = 0; j < NPT; j++)
            if (act[j]) {
                E[j] += a.Pc ? dts[j] * R[j] / Cp[j] : dts[j] * R[j];
                a.Esh[base + (int64_t)j * NT] = E[j];
            }
    }
#pragma unroll
    for (int j = 0; j < NPT; j++)
        if (act[j])
            for (int k = k0[j]; k < k1[j]; ++k) {
                const int32_t mp = __ldg(a.mpos + k);
                if (FEM_IN(mp, (int64_t)a.n_blocks * a.ls, a.err)) a.Eloc[mp] = E[j];
            }
}

// Interface faces (Eq. 8): every interface face is a Robin face whose
// ambient temperature is the mean temperature of its sister face (the
// nearest face of the other region, Section 3) at step n.  This kernel
// writes the face's load term A/3 h_i T_sister into the face arrays before
// the step's element pass; its h_i A / 12 matrix term is static.
template <typename real>
__global__ void k_interface(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                            const real *ranges, real *fg, const int32_t *pos, const int32_t *sis,
                            const real *g, int64_t n)
{
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < n;
         f += (int64_t)gridDim.x * blockDim.x) {
        real T = real(0);
#pragma unroll
        for (int c = 0; c < 3; c++) {
            const int32_t i = sis[3 * f + c];
            T += state_T(v, i);
        }
        fg[pos[f]] = g[f] * (T / real(3));
    }
}

// ---------------------------------------------------------------------------
// Flat variants (atomic / coloured), for comparison
// ---------------------------------------------------------------------------
template <typename real>
__global__ void k_flat_temperature(const FlatArgs<real> a)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n_nodes;
         i += (int64_t)gridDim.x * blockDim.x) {
        a.T[i] = temperature_of(a.E[i], __ldg(a.C + i), __ldg(a.Lc + i), __ldg(a.ph + i), a.ranges);
        a.R[i] = real(0);
    }
}

template <typename real, bool kAtomic, bool KT>
__global__ void k_flat_elements(const FlatArgs<real> a, const int64_t p0, const int64_t p1)
{
    const int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int64_t st = a.e_stride;
    const int32_t n0 = __ldg(a.conn + p);
    if (n0 < 0) return;   // padding
    const int32_t n1 = __ldg(a.conn + st + p), n2 = __ldg(a.conn + 2 * st + p),
                  n3 = __ldg(a.conn + 3 * st + p);
    if (!FEM_IN(n0, a.n_nodes, a.err) || !FEM_IN(n1, a.n_nodes, a.err) ||
        !FEM_IN(n2, a.n_nodes, a.err) || !FEM_IN(n3, a.n_nodes, a.err))
        return;
    const real T0 = __ldg(a.T + n0), T1 = __ldg(a.T + n1), T2 = __ldg(a.T + n2), T3 = __ldg(a.T + n3);
    real kk = real(1);
    if (KT)   // K^e(T) = k(mean element temperature) x the k = 1 weights
        kk = conductivity_of(a.kt_T, a.kt_k, a.kt_n, (int)__ldg(a.emat + p),
                             (T0 + T1 + T2 + T3) * real(0.25));
    const real p01 = (kk * __ldg(a.w + p)) * (T1 - T0), p02 = (kk * __ldg(a.w + st + p)) * (T2 - T0),
               p03 = (kk * __ldg(a.w + 2 * st + p)) * (T3 - T0);
    const real p12 = (kk * __ldg(a.w + 3 * st + p)) * (T2 - T1),
               p13 = (kk * __ldg(a.w + 4 * st + p)) * (T3 - T1),
               p23 = (kk * __ldg(a.w + 5 * st + p)) * (T3 - T2);
    const real r0 = p01 + p02 + p03, r1 = (p12 + p13) - p01, r2 = p23 - (p02 + p12),
               r3 = -(p03 + p13 + p23);
    if (kAtomic) {
        atomicAdd(a.R + n0, r0);
        atomicAdd(a.R + n1, r1);
        atomicAdd(a.R + n2, r2);
        atomicAdd(a.R + n3, r3);
    } else {   // one colour: no two elements of this launch share a node
        a.R[n0] += r0;
        a.R[n1] += r1;
        a.R[n2] += r2;
        a.R[n3] += r3;
    }
}

// Node update with the Robin faces gathered per node (node -> faces CSR).
template <typename real, int NT>
__global__ void __launch_bounds__(NT) k_flat_update(const FlatArgs<real> a, const int32_t *nf_ptr,
                                                    const int32_t *nf_idx, const real dt)
{
    const int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x;
    double acc[1] = {0.0};
    if (i < a.n_nodes) {
        real R = a.R[i];
        const real Ti = a.T[i];
        const int32_t f1 = __ldg(nf_ptr + i + 1);
        for (int32_t k = __ldg(nf_ptr + i); k < f1; ++k) {
            const int32_t f = __ldg(nf_idx + k);
            const int64_t fs = a.f_stride;
            const real S = __ldg(a.T + __ldg(a.fconn + f)) + __ldg(a.T + __ldg(a.fconn + fs + f)) +
                           __ldg(a.T + __ldg(a.fconn + 2 * fs + f));
            const real r = __ldg(a.fg + f) - __ldg(a.fa + f) * (Ti + S);
            R += r;
            acc[0] += (double)r;
        }
        if (!(__ldg(a.ph + i) & kDirichletBit)) a.E[i] += dt * R;
    }
    block_sum<NT, 1>(acc);
    if (threadIdx.x == 0) a.qcum[blockIdx.x] += (double)dt * acc[0];
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
// The block kernel instantiation for (threads, kt), as a function pointer.
template <typename real>
using BlockKernel = void (*)(const BlockArgs<real>, const real);
template <typename real, int NT>
BlockKernel<real> block_kernel_nt(bool kt, bool lm)
{
    if (lm) return kt ? k_block_step<real, NT, true, true> : k_block_step<real, NT, false, true>;
    return kt ? k_block_step<real, NT, true, false> : k_block_step<real, NT, false, false>;
}
template <typename real>
BlockKernel<real> block_kernel_for(int threads, bool kt, bool lm, bool wg)
{
    if (wg) {   // enthalpy formulation only (the apparent capacity keeps its
                // element capacities over the staged conductance rows)
        if (lm || threads != 256) return nullptr;
        return kt ? k_block_step<real, 256, true, false, true> : k_block_step<real, 256, false, false, true>;
    }
    switch (threads) {
    case 128: return block_kernel_nt<real, 128>(kt, lm);
    case 256: return block_kernel_nt<real, 256>(kt, lm);
    case 512: return block_kernel_nt<real, 512>(kt, lm);
    case 1024: return block_kernel_nt<real, 1024>(kt, lm);
    default: return nullptr;
    }
}

template <typename real>
int block_kernel_occupancy(int threads, size_t smem_bytes, int *ctas_per_sm, bool kt, bool lm, bool wg)
{
    BlockKernel<real> f = block_kernel_for<real>(threads, kt, lm, wg);
    if (!f) return (int)cudaErrorInvalidValue;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, f, threads, smem_bytes);
}

template <typename real>
int configure_block_kernel(int threads, size_t smem_bytes, bool kt, bool lm, bool wg)
{
    BlockKernel<real> f = block_kernel_for<real>(threads, kt, lm, wg);
    if (!f) return (int)cudaErrorInvalidValue;
    return (int)cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_bytes);
}

template <typename real>
int launch_block_kernel(const BlockArgs<real> &a, int threads, size_t smem_bytes, double dt,
                        void *stream, bool kt, bool lm, bool wg)
{
    const int grid = a.b_count;
    if (grid <= 0) return 0;
    BlockKernel<real> f = block_kernel_for<real>(threads, kt, lm, wg);
    if (!f) return (int)cudaErrorInvalidValue;
    f<<<grid, threads, smem_bytes, (cudaStream_t)stream>>>(a, (real)dt);
    return (int)cudaGetLastError();
}

constexpr int kShNT = 256, kShNPT = 2;   // exchange kernel: threads, nodes per thread

template <typename real>
int launch_interface(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                     const real *ranges, real *fg, const int32_t *pos, const int32_t *sis,
                     const real *g, int64_t n, void *stream)
{
    if (n > 0)
        k_interface<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, C, Lc, ph, ranges, fg,
                                                                           pos, sis, g, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_mirror_copies(const BlockArgs<real> &a, void *stream)
{
    const int64_t n = a.s_end - a.s_first, per = (int64_t)kShNT * kShNPT;
    if (n > 0)
        k_shared_update<real, kShNT, kShNPT><<<(int)((n + per - 1) / per), kShNT, 0,
                                               (cudaStream_t)stream>>>(a, real(0), false);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_shared_update(const BlockArgs<real> &a, double dt, void *stream)
{
    const int64_t n = a.s_end - a.s_first, per = (int64_t)kShNT * kShNPT;
    if (n > 0)
        k_shared_update<real, kShNT, kShNPT><<<(int)((n + per - 1) / per), kShNT, 0,
                                               (cudaStream_t)stream>>>(a, (real)dt, true);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_flat_temperature(const FlatArgs<real> &a, void *stream)
{
    k_flat_temperature<real><<<grid_for(a.n_nodes, 256), 256, 0, (cudaStream_t)stream>>>(a);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_flat_elements(const FlatArgs<real> &a, bool atomic, const int64_t *color_start,
                         int n_colors, void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const bool kt = a.emat != nullptr;
    if (atomic) {
        const int64_t ne = a.e_stride;
        if (kt)
            k_flat_elements<real, true, true><<<(int)((ne + 255) / 256), 256, 0, st>>>(a, 0, ne);
        else
            k_flat_elements<real, true, false><<<(int)((ne + 255) / 256), 256, 0, st>>>(a, 0, ne);
    } else {
        for (int c = 0; c < n_colors; c++) {
            const int64_t p0 = color_start[c], p1 = color_start[c + 1];
            if (p1 <= p0) continue;
            if (kt)
                k_flat_elements<real, false, true><<<(int)((p1 - p0 + 255) / 256), 256, 0, st>>>(a, p0, p1);
            else
                k_flat_elements<real, false, false><<<(int)((p1 - p0 + 255) / 256), 256, 0, st>>>(a, p0, p1);
        }
    }
    return (int)cudaGetLastError();
}

template <typename real>
int launch_flat_update(const FlatArgs<real> &a, const int32_t *nf_ptr, const int32_t *nf_idx,
                       int n_node_ctas, double dt, void *stream)
{
    k_flat_update<real, 256><<<n_node_ctas, 256, 0, (cudaStream_t)stream>>>(a, nf_ptr, nf_idx, (real)dt);
    return (int)cudaGetLastError();
}

#define FEM_INSTANTIATE(real)                                                                     \
    template int configure_block_kernel<real>(int, size_t, bool, bool, bool);                     \
    template int block_kernel_occupancy<real>(int, size_t, int *, bool, bool, bool);              \
    template int launch_mirror_copies<real>(const BlockArgs<real> &, void *);                     \
    template int launch_interface<real>(StateView<real>, const real *, const real *,              \
                                        const uint8_t *, const real *, real *, const int32_t *,   \
                                        const int32_t *, const real *, int64_t, void *);          \
    template int launch_block_kernel<real>(const BlockArgs<real> &, int, size_t, double, void *,  \
                                           bool, bool, bool);                                     \
    template int launch_shared_update<real>(const BlockArgs<real> &, double, void *);             \
    template int launch_flat_temperature<real>(const FlatArgs<real> &, void *);                   \
    template int launch_flat_elements<real>(const FlatArgs<real> &, bool, const int64_t *, int,  \
                                            void *);                                              \
    template int launch_flat_update<real>(const FlatArgs<real> &, const int32_t *,                \
                                          const int32_t *, int, double, void *);

FEM_INSTANTIATE(float)
FEM_INSTANTIATE(double)

}  // namespace fem
