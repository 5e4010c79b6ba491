// CUDA kernels of libfem for sm_103a: one explicit EBE enthalpy step
// (Eq. 14 in the enthalpy form of Eq. 5, element sums of Eqs. 15-22) and
// the small kernels around it (initial state, read-back, FP64 energy).
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
// are FP64 reductions of the state (k_energy_snapshot) taken on demand.
#include <cuda_runtime.h>

#include <cstdint>

#include "fem_internal.h"

namespace fem {

namespace {

// Temperature of a node from its enthalpy content E (J): the inverse of
// E(T) = C T + Lc f_l(T), f_l linear between Ts and Tl (Eqs. 5, 11).
template <typename real>
__device__ __forceinline__ real temperature_of(real E, real C, real Lc, uint8_t ph,
                                               const real *__restrict__ ranges)
{
    if (!(Lc > real(0))) return E / C;
    const int r = ph & 0x7F;
    const real Ts = __ldg(ranges + 2 * r), Tl = __ldg(ranges + 2 * r + 1);
    const real E_sol = C * Ts;            // fully solid at the solidus
    if (E <= E_sol) return E / C;
    const real E_liq = C * Tl + Lc;       // fully liquid at the liquidus
    if (E >= E_liq) return (E - Lc) / C;
    if (Tl <= Ts) return Ts;              // isothermal plateau
    return Ts + (E - E_sol) / (C + Lc / (Tl - Ts));
}

// Enthalpy content of a node at temperature T.
template <typename real>
__device__ __forceinline__ real enthalpy_of(real T, real C, real Lc, uint8_t ph,
                                            const real *__restrict__ ranges)
{
    if (!(Lc > real(0))) return C * T;
    const int r = ph & 0x7F;
    const real Ts = __ldg(ranges + 2 * r), Tl = __ldg(ranges + 2 * r + 1);
    real fl;
    if (Tl <= Ts) fl = T >= Ts ? real(1) : real(0);
    else fl = T <= Ts ? real(0) : (T >= Tl ? real(1) : (T - Ts) / (Tl - Ts));
    return C * T + Lc * fl;
}

// Latent heat still held by a node: E - C T(E), in [0, Lc].
template <typename real>
__device__ __forceinline__ double latent_of(real E, real C, real Lc, uint8_t ph,
                                            const real *__restrict__ ranges)
{
    if (!(Lc > real(0))) return 0.0;
    const real T = temperature_of(E, C, Lc, ph, ranges);
    double l = (double)E - (double)C * (double)T;
    return l < 0.0 ? 0.0 : (l > (double)Lc ? (double)Lc : l);
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Deterministic block sum of K doubles per thread; result valid in thread 0.
template <int NT, int K>
__device__ __forceinline__ void block_sum(double (&v)[K])
{
    __shared__ double red[NT / 32][K];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; k++) v[k] = warp_sum(v[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) red[warp][k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double s = 0.0;
            for (int w = 0; w < NT / 32; w++) s += red[w][k];
            v[k] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Block variant
// ---------------------------------------------------------------------------

// PTX wrappers: mbarrier + 1-D bulk copy (TMA) global -> shared.
__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_load(uint32_t dst, const void *src, uint32_t bytes, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}
// Waits for phase `parity` of the barrier; gives up after kSpinLimit polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    for (uint32_t i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
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

// One CTA per element block.  Thread t owns local nodes t, t+NT, ... in
// every pass (32-lane group g = warp + j*NW covers nodes 32 g + lane), so
// their T and E stay in registers.
template <typename real, int NT>
__global__ void __launch_bounds__(NT, 2) k_block_step(const BlockArgs<real> a, const real dt)
{
    constexpr int NW = NT / 32;
    constexpr int MAXJ = kMaxLocalNodes / NT;   // local nodes per thread
    using V = typename Vec4Of<real>::type;
    constexpr int VN = Vec4Of<real>::n;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    const BlockInfo bi = a.blocks[blockIdx.x];
    const int nloc = bi.nint + bi.nsh;
    const int ne_pad = bi.ne_pad, nf_pad = bi.nf_pad, nep = bi.nep;
    const int dummy = 4 * ne_pad + 3 * nf_pad;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // shared memory: [barriers][weights][schedule][slots + dummy]
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem_raw);
    unsigned char *q = smem_raw + kSmemBarBytes;
    real *sw = reinterpret_cast<real *>(q);
    q += align16(6 * (size_t)nep * sizeof(real));
    const uint32_t *ss = reinterpret_cast<const uint32_t *>(q);   // [pair][lane]
    q += align16((size_t)bi.nrounds * 64);
    real *sv = reinterpret_cast<real *>(q);
    const uint32_t bar_s = smem_addr(&bars[0]), bar_w = smem_addr(&bars[1]);

    // bulk copies: the block's schedule and its six conductance rows
    if (threadIdx.x == 0) {
        mbar_init(bar_s, 1);
        mbar_init(bar_w, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t sbytes = (uint32_t)bi.nrounds * 64u;
        mbar_arrive_expect_tx(bar_s, sbytes);
        if (sbytes) bulk_load(smem_addr(ss), a.sched + (size_t)bi.r0 * 32, sbytes, bar_s);
        const uint32_t wbytes = (uint32_t)(6 * (size_t)nep * sizeof(real));
        mbar_arrive_expect_tx(bar_w, wbytes);
        bulk_load(smem_addr(sw), a.w + 6 * (size_t)bi.e0, wbytes, bar_w);
    }

    // nodal enthalpy -> temperature (Eqs. 5, 11), overlapping the copies
    real Tl[MAXJ], El[MAXJ];
#pragma unroll
    for (int j = 0; j < MAXJ; j++) {
        const int l = threadIdx.x + j * NT;
        Tl[j] = real(0);
        El[j] = real(0);
        if (l < nloc) {
            const int64_t gid = l < bi.nint ? (int64_t)bi.n0 + l
                                            : (int64_t)__ldg(a.copy_node + bi.c0 + (l - bi.nint));
            El[j] = a.E[gid];
            Tl[j] = temperature_of(El[j], __ldg(a.C + gid), __ldg(a.Lc + gid), __ldg(a.ph + gid),
                                   a.ranges);
        }
    }

    // one thread polls (bounded), then every thread observes the phase
    int failed = 0;
    if (threadIdx.x == 0) failed = !mbar_wait(bar_s, 0);
    if (__syncthreads_or(failed)) goto timeout;
    mbar_try_wait(bar_s, 0);

    // pass 1: T of every local node into the slots of its element corners
    // (padding entries all name the dummy slot)
#pragma unroll
    for (int j = 0; j < MAXJ; j++) {
        const int g = warp + j * NW;
        if (g < bi.ngrp) {
            const int p0 = (__ldg(a.grp + bi.g0 + g) - bi.r0) >> 1;
            const int p1 = (__ldg(a.grp + bi.g0 + g + 1) - bi.r0) >> 1;
            const real T = Tl[j];
            for (int pr = p0; pr < p1; ++pr) {
                const uint32_t v = ss[pr * 32 + lane];
                sv[v & 0xFFFFu] = T;
                sv[v >> 16] = T;
            }
        }
    }
    if (threadIdx.x == 0) failed = !mbar_wait(bar_w, 0);
    if (__syncthreads_or(failed)) goto timeout;
    mbar_try_wait(bar_w, 0);

    // pass 2: element products, VN elements per 16-byte access
    for (int e = threadIdx.x * VN; e < bi.ne; e += NT * VN) {
        const V w01 = *reinterpret_cast<const V *>(sw + e);
        const V w02 = *reinterpret_cast<const V *>(sw + nep + e);
        const V w03 = *reinterpret_cast<const V *>(sw + 2 * nep + e);
        const V w12 = *reinterpret_cast<const V *>(sw + 3 * nep + e);
        const V w13 = *reinterpret_cast<const V *>(sw + 4 * nep + e);
        const V w23 = *reinterpret_cast<const V *>(sw + 5 * nep + e);
        V T0 = *reinterpret_cast<const V *>(sv + e);
        V T1 = *reinterpret_cast<const V *>(sv + ne_pad + e);
        V T2 = *reinterpret_cast<const V *>(sv + 2 * ne_pad + e);
        V T3 = *reinterpret_cast<const V *>(sv + 3 * ne_pad + e);
#pragma unroll
        for (int i = 0; i < VN; i++) {
            V c01 = w01, c02 = w02, c03 = w03, c12 = w12, c13 = w13, c23 = w23;
            tet_products(vat(c01, i), vat(c02, i), vat(c03, i), vat(c12, i), vat(c13, i),
                         vat(c23, i), vat(T0, i), vat(T1, i), vat(T2, i), vat(T3, i), vat(T0, i),
                         vat(T1, i), vat(T2, i), vat(T3, i));
        }
        *reinterpret_cast<V *>(sv + e) = T0;
        *reinterpret_cast<V *>(sv + ne_pad + e) = T1;
        *reinterpret_cast<V *>(sv + 2 * ne_pad + e) = T2;
        *reinterpret_cast<V *>(sv + 3 * ne_pad + e) = T3;
    }
    if (threadIdx.x == 0) sv[dummy] = real(0);   // padding adds nothing in pass 3
    // Robin faces (Eq. 4): r_c = A/3 (h T_inf - q) - h A/12 (T_c + T_0 + T_1 + T_2)
    {
        double qin = 0.0;   // heat entering through the block's faces (FP64)
        const int fbase = 4 * ne_pad;
        for (int f = threadIdx.x; f < bi.nf; f += NT) {
            real *s0 = sv + fbase + f;
            const real T0 = s0[0], T1 = s0[nf_pad], T2 = s0[2 * nf_pad];
            const real ha = __ldg(a.fa + bi.f0 + f), hg = __ldg(a.fg + bi.f0 + f);
            const real S = T0 + T1 + T2;
            const real r0 = hg - ha * (T0 + S), r1 = hg - ha * (T1 + S), r2 = hg - ha * (T2 + S);
            s0[0] = r0;
            s0[nf_pad] = r1;
            s0[2 * nf_pad] = r2;
            qin += (double)r0 + (double)r1 + (double)r2;
        }
        __syncthreads();

        // pass 3: fixed-order node sums; interior update or shared partial
#pragma unroll
        for (int j = 0; j < MAXJ; j++) {
            const int g = warp + j * NW;
            if (g >= bi.ngrp) continue;
            const int l = 32 * g + lane;
            const int p0 = (__ldg(a.grp + bi.g0 + g) - bi.r0) >> 1;
            const int p1 = (__ldg(a.grp + bi.g0 + g + 1) - bi.r0) >> 1;
            real R = real(0);
            for (int pr = p0; pr < p1; ++pr) {
                const uint32_t v = ss[pr * 32 + lane];
                R += sv[v & 0xFFFFu];
                R += sv[v >> 16];
            }
            if (l < bi.nint) {
                const int64_t gid = (int64_t)bi.n0 + l;
                if (!(__ldg(a.ph + gid) & kDirichletBit)) a.E[gid] = El[j] + dt * R;
            } else if (l < nloc) {
                a.P[__ldg(a.copy_pos + bi.c0 + (l - bi.nint))] = R;
            }
        }
        // cumulative boundary heat of the blocks that own Robin faces
        if (bi.nf > 0) {
            double acc[1] = {qin};
            block_sum<NT, 1>(acc);
            if (threadIdx.x == 0) a.qcum[blockIdx.x] += (double)dt * acc[0];
        }
    }
    return;

timeout:
    // a copy did not complete in time: flag it, give the copies in flight a
    // bounded second chance to land before the shared memory is released
    if (threadIdx.x == 0) {
        atomicExch(a.err, kErrWaitTimeout);
        mbar_wait(bar_s, 0);
        mbar_wait(bar_w, 0);
    }
    __syncthreads();
}

template <typename real, int NT>
__global__ void __launch_bounds__(NT) k_shared_update(const BlockArgs<real> a, const int64_t n_sh,
                                                      const real dt)
{
    const int64_t s = (int64_t)blockIdx.x * NT + threadIdx.x;
    if (s >= n_sh) return;
    const int64_t gid = a.n_int + s;
    if (__ldg(a.ph + gid) & kDirichletBit) return;
    real R = real(0);
    const int k1 = __ldg(a.sh_ptr + s + 1);
    for (int k = __ldg(a.sh_ptr + s); k < k1; ++k) R += a.P[k];   // block order
    a.E[gid] += dt * R;
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

template <typename real, bool kAtomic>
__global__ void k_flat_elements(const FlatArgs<real> a, const int64_t p0, const int64_t p1)
{
    const int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= p1) return;
    const int64_t st = a.e_stride;
    const int32_t n0 = __ldg(a.conn + p);
    if (n0 < 0) return;   // padding
    const int32_t n1 = __ldg(a.conn + st + p), n2 = __ldg(a.conn + 2 * st + p),
                  n3 = __ldg(a.conn + 3 * st + p);
    const real T0 = __ldg(a.T + n0), T1 = __ldg(a.T + n1), T2 = __ldg(a.T + n2), T3 = __ldg(a.T + n3);
    const real p01 = __ldg(a.w + p) * (T1 - T0), p02 = __ldg(a.w + st + p) * (T2 - T0),
               p03 = __ldg(a.w + 2 * st + p) * (T3 - T0);
    const real p12 = __ldg(a.w + 3 * st + p) * (T2 - T1), p13 = __ldg(a.w + 4 * st + p) * (T3 - T1),
               p23 = __ldg(a.w + 5 * st + p) * (T3 - T2);
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

// ---------------------------------------------------------------------------
// State I/O and energy
// ---------------------------------------------------------------------------
template <typename real>
__global__ void k_set_temperature(real *E, const real *C, const real *Lc, const uint8_t *ph,
                                  const real *ranges, const double *T_in, const int32_t *node_old,
                                  const double *dirT_int, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t p = ph[i];
        const double T = (dirT_int && (p & kDirichletBit)) ? dirT_int[i] : T_in[node_old[i]];
        E[i] = enthalpy_of((real)T, C[i], Lc[i], p, ranges);
    }
}

template <typename real>
__global__ void k_set_state(real *E, const double *E_in, const int32_t *node_old, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        E[i] = (real)E_in[node_old[i]];
}

template <typename real>
__global__ void k_get_temperature(const real *E, const real *C, const real *Lc, const uint8_t *ph,
                                  const real *ranges, double *T_out, const int32_t *node_old,
                                  int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        T_out[node_old[i]] = (double)temperature_of(E[i], C[i], Lc[i], ph[i], ranges);
}

template <typename real>
__global__ void k_get_state(const real *E, double *E_out, const int32_t *node_old, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        E_out[node_old[i]] = (double)E[i];
}

template <typename real, int NT>
__global__ void __launch_bounds__(NT) k_energy_snapshot(const real *E, const real *C, const real *Lc,
                                                        const uint8_t *ph, const real *ranges,
                                                        int64_t n, double *part)
{
    double acc[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        acc[0] += (double)E[i];
        acc[1] += latent_of(E[i], C[i], Lc[i], ph[i], ranges);
    }
    block_sum<NT, 2>(acc);
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = acc[0];
        part[2 * blockIdx.x + 1] = acc[1];
    }
}

constexpr int kReduceThreads = 1024;

__global__ void __launch_bounds__(kReduceThreads) k_energy_reduce(const double *pa, int64_t na,
                                                                  const double *pb, int64_t nb,
                                                                  const double *q, int64_t nq,
                                                                  double *out)
{
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t i = threadIdx.x; i < na; i += kReduceThreads) {
        acc[0] += pa[2 * i];
        acc[1] += pa[2 * i + 1];
    }
    for (int64_t i = threadIdx.x; i < nb; i += kReduceThreads) {
        acc[0] += pb[2 * i];
        acc[1] += pb[2 * i + 1];
    }
    for (int64_t i = threadIdx.x; i < nq; i += kReduceThreads) acc[2] += q[i];
    block_sum<kReduceThreads, 3>(acc);
    if (threadIdx.x == 0) {
        out[0] = acc[0];
        out[1] = acc[1];
        out[2] = acc[2];
    }
}

inline int grid_for(int64_t n, int threads)
{
    int64_t g = (n + threads - 1) / threads;
    if (g > 152 * 64) g = 152 * 64;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <typename real>
int configure_block_kernel(int threads, size_t smem_bytes)
{
    cudaError_t e = cudaSuccess;
    const int s = (int)smem_bytes;
    switch (threads) {
    case 128: e = cudaFuncSetAttribute(k_block_step<real, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize, s); break;
    case 256: e = cudaFuncSetAttribute(k_block_step<real, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize, s); break;
    case 512: e = cudaFuncSetAttribute(k_block_step<real, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize, s); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)e;
}

template <typename real>
int launch_block_kernel(const BlockArgs<real> &a, int threads, size_t smem_bytes, double dt,
                        void *stream)
{
    cudaStream_t st = (cudaStream_t)stream;
    const real rdt = (real)dt;
    switch (threads) {
    case 128: k_block_step<real, 128><<<a.n_blocks, 128, smem_bytes, st>>>(a, rdt); break;
    case 256: k_block_step<real, 256><<<a.n_blocks, 256, smem_bytes, st>>>(a, rdt); break;
    case 512: k_block_step<real, 512><<<a.n_blocks, 512, smem_bytes, st>>>(a, rdt); break;
    default: return (int)cudaErrorInvalidValue;
    }
    return (int)cudaGetLastError();
}

template <typename real>
int launch_shared_update(const BlockArgs<real> &a, int64_t n_sh, int n_sh_ctas, double dt,
                         void *stream)
{
    if (n_sh > 0)
        k_shared_update<real, 256><<<n_sh_ctas, 256, 0, (cudaStream_t)stream>>>(a, n_sh, (real)dt);
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
    if (atomic) {
        const int64_t ne = a.e_stride;
        k_flat_elements<real, true><<<(int)((ne + 255) / 256), 256, 0, st>>>(a, 0, ne);
    } else {
        for (int c = 0; c < n_colors; c++) {
            const int64_t p0 = color_start[c], p1 = color_start[c + 1];
            if (p1 > p0)
                k_flat_elements<real, false><<<(int)((p1 - p0 + 255) / 256), 256, 0, st>>>(a, p0, p1);
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

template <typename real>
int launch_set_temperature(real *E, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, const double *T_in, const int32_t *node_old,
                           const double *dirT_int, int64_t n, void *stream)
{
    k_set_temperature<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        E, C, Lc, ph, ranges, T_in, node_old, dirT_int, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_set_state(real *E, const double *E_in, const int32_t *node_old, int64_t n, void *stream)
{
    k_set_state<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(E, E_in, node_old, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_get_temperature(const real *E, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, double *T_out, const int32_t *node_old, int64_t n,
                           void *stream)
{
    k_get_temperature<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        E, C, Lc, ph, ranges, T_out, node_old, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_get_state(const real *E, double *E_out, const int32_t *node_old, int64_t n, void *stream)
{
    k_get_state<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(E, E_out, node_old, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_energy_snapshot(const real *E, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, int64_t n, double *part, int n_ctas, void *stream)
{
    k_energy_snapshot<real, 256><<<n_ctas, 256, 0, (cudaStream_t)stream>>>(E, C, Lc, ph, ranges, n, part);
    return (int)cudaGetLastError();
}

int launch_energy_reduce(const double *pa, int64_t na, const double *pb, int64_t nb, const double *q,
                         int64_t nq, double *out, void *stream)
{
    k_energy_reduce<<<1, kReduceThreads, 0, (cudaStream_t)stream>>>(pa, na, pb, nb, q, nq, out);
    return (int)cudaGetLastError();
}

#define FEM_INSTANTIATE(real)                                                                     \
    template int configure_block_kernel<real>(int, size_t);                                       \
    template int launch_block_kernel<real>(const BlockArgs<real> &, int, size_t, double, void *); \
    template int launch_shared_update<real>(const BlockArgs<real> &, int64_t, int, double, void *); \
    template int launch_flat_temperature<real>(const FlatArgs<real> &, void *);                   \
    template int launch_flat_elements<real>(const FlatArgs<real> &, bool, const int64_t *, int,  \
                                            void *);                                              \
    template int launch_flat_update<real>(const FlatArgs<real> &, const int32_t *,                \
                                          const int32_t *, int, double, void *);                  \
    template int launch_set_temperature<real>(real *, const real *, const real *,                 \
                                              const uint8_t *, const real *, const double *,      \
                                              const int32_t *, const double *, int64_t, void *);  \
    template int launch_set_state<real>(real *, const double *, const int32_t *, int64_t, void *); \
    template int launch_get_temperature<real>(const real *, const real *, const real *,           \
                                              const uint8_t *, const real *, double *,            \
                                              const int32_t *, int64_t, void *);                  \
    template int launch_get_state<real>(const real *, double *, const int32_t *, int64_t, void *); \
    template int launch_energy_snapshot<real>(const real *, const real *, const real *,           \
                                              const uint8_t *, const real *, int64_t, double *,   \
                                              int, void *);

FEM_INSTANTIATE(float)
FEM_INSTANTIATE(double)

}  // namespace fem
