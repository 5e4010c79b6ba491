// Launchers of the state I/O and energy kernels (fem_io.cu): the
// permutations between the caller's node order and the step kernels' layout
// and the FP64 energy sums.  Host-callable; all pointers are device pointers
// except where noted, and every launcher returns a cudaError_t value (0 on
// success).
#pragma once

#include "fem_internal.h"

namespace fem {

// Initial state / read-back kernels (any variant, through a StateView).
template <typename real>
int launch_set_temperature(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, const double *T_in, const int32_t *node_old,
                           const double *dirT_int, int64_t n, void *stream);
// launch_set_state / launch_get_temperature set kErrBadInput / kErrNonFinite
// in *err for non-finite values (err may be null).  With sh_ptr and mpos
// (block variant: shared node -> copies, copy -> mirror position, n_loc
// entries of the local arrays) the set-state kernels also write the shared
// nodes' mirrors.
template <typename real>
int launch_set_state(StateView<real> v, const double *E_in, const int32_t *node_old, int64_t n,
                     int *err, void *stream, const int32_t *sh_ptr = nullptr,
                     const int32_t *mpos = nullptr, int64_t n_loc = 0);
// (The read-back takes C, Lc, the phase bytes and the ranges from the view;
// the C, Lc, ph and ranges arguments are not used.)
template <typename real>
int launch_get_temperature(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, double *T_out, const int32_t *node_old, int64_t n,
                           int *err, void *stream);
// The same with the caller's arrays in FP32 (fem_set_state_async_f32,
// fem_get_temperature_async_f32).
template <typename real>
int launch_set_state_f32(StateView<real> v, const float *E_in, const int32_t *node_old, int64_t n,
                         int *err, void *stream, const int32_t *sh_ptr = nullptr,
                         const int32_t *mpos = nullptr, int64_t n_loc = 0);
template <typename real>
int launch_get_temperature_f32(StateView<real> v, const real *ranges, float *T_out,
                               const int32_t *node_old, int64_t n, int *err, void *stream);
template <typename real>
int launch_get_state(StateView<real> v, double *E_out, const int32_t *node_old, int64_t n,
                     void *stream);
template <typename real>
int launch_energy_snapshot(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, int64_t n, double *part, int n_ctas, void *stream);
// Sums n_a pairs of part_a, n_b pairs of part_b and n_q entries of q into
// out[0] (sum E), out[1] (latent), out[2] (boundary heat).
int launch_energy_reduce(const double *part_a, int64_t n_a, const double *part_b, int64_t n_b,
                         const double *q, int64_t n_q, double *out, void *stream);

}  // namespace fem
