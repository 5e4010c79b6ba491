// Device helpers shared by the CUDA translation units of libfem (device
// code only): the nodal phase-change relations of the enthalpy formulation
// (Eqs. 5 and 11 with a linear liquid fraction between the solidus Ts and
// the liquidus Tl: E(T) = C T + Lc f_l(T) and its exact piecewise-linear
// inverse T(E)), and PTX wrappers for mbarriers and bulk copies.
#pragma once

#include <cstdint>

#include "fem_internal.h"

namespace fem {

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

// The same from the reciprocal capacity rC = 1/C (rounded once): the solid
// and liquid branches become products, and only the mushy branch divides.
// Ta = E / C is the temperature if no latent heat were stored, Tb the
// temperature if all of it were; T(E) is Ta below the solidus, Tb above the
// liquidus and, in between, the point where E = C T + Lc (T - Ts)/(Tl - Ts).
template <typename real>
__device__ __forceinline__ real temperature_of_rc(real E, real rC, real Lc, uint8_t ph,
                                                  const real *__restrict__ ranges)
{
    const real Ta = E * rC;
    if (!(Lc > real(0))) return Ta;
    const int r = ph & 0x7F;
    const real Ts = __ldg(ranges + 2 * r), Tl = __ldg(ranges + 2 * r + 1);
    if (Ta <= Ts) return Ta;
    const real Tb = (E - Lc) * rC;
    if (Tb >= Tl) return Tb;
    if (Tl <= Ts) return Ts;   // isothermal plateau
    return Ts + (Ta - Ts) / (real(1) + Lc * rC / (Tl - Ts));
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
// Bulk prefetch of [src, src + bytes) into L2 (16-byte aligned address and
// size; nothing to wait for).
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
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
__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Waits for phase `parity` of the barrier; gives up after kWaitNs of device
// time or kWaitPolls polls.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    for (uint32_t i = 1; i < kWaitPolls; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 63u) == 0 && global_ns() - t0 > kWaitNs) return false;
    }
    return false;
}

}  // namespace fem
