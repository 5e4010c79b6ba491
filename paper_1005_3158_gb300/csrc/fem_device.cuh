// Nodal phase-change relations of the enthalpy formulation, shared by the
// CUDA translation units of libfem (device code only).  Eqs. 5 and 11 with a
// linear liquid fraction between the solidus Ts and the liquidus Tl:
// E(T) = C T + Lc f_l(T) and its exact piecewise-linear inverse T(E).
#pragma once

#include <cstdint>

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

}  // namespace fem
