// State I/O and energy kernels of libfem: the permutations between the
// caller's node order and the layout of the step kernels (initial state,
// upload of a state, read-back of T or E) and the FP64 energy sums taken on
// demand (Sigma E and the latent heat still held, from the state).
#include <cuda_runtime.h>

#include <cstdint>

#include "fem_io.h"
#include "fem_state.cuh"

namespace fem {

namespace {

template <typename real>
__global__ void k_set_temperature(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                                  const real *ranges, const double *T_in, const int32_t *node_old,
                                  const double *dirT_int, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint8_t p = ph[i];
        const double T = (dirT_int && (p & kDirichletBit)) ? dirT_int[i] : T_in[node_old[i]];
        state_set_T(v, i, (real)T);
    }
}

// io: the element type of the caller's array (double, or float for the
// FP32 host I/O of fem_set_state_async_f32 / fem_get_temperature_async_f32).
// The upload takes kIoBatch nodes per thread per round, grid-stride apart,
// all loads first: their index -> value -> store chains then overlap
// instead of running one after another.
constexpr int kIoBatch = 4;

// With sh_ptr / mpos (block variant), a shared node's mirrors in the
// blocks' local arrays are written too, so that no separate mirror refresh
// has to follow.
template <typename real, typename io = double>
__global__ void k_set_state(StateView<real> v, const io *E_in, const int32_t *node_old, int64_t n,
                            int *err, const int32_t *sh_ptr, const int32_t *mpos, int64_t n_loc)
{
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < n; i0 += kIoBatch * stride) {
        double E[kIoBatch];
#pragma unroll
        for (int u = 0; u < kIoBatch; u++) {
            const int64_t i = i0 + u * stride;
            E[u] = i < n ? (double)E_in[node_old[i]] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < kIoBatch; u++) {
            const int64_t i = i0 + u * stride;
            if (i < n) {
                bad |= !isfinite(E[u]);
                state_set_E(v, i, (real)E[u]);
                if (sh_ptr && i >= v.n_int) {
                    const int64_t sn = i - v.n_int;
                    const real stored = v.Esh[sn];
                    const int k1 = __ldg(sh_ptr + sn + 1);
                    for (int k = __ldg(sh_ptr + sn); k < k1; ++k) {
                        const int32_t mp = __ldg(mpos + k);
                        if (FEM_IN(mp, n_loc, err)) v.Eloc[mp] = stored;
                    }
                }
            }
        }
    }
    if (bad && err) atomicOr(err, kErrBadInput);
}

// Four consecutive entries of a node array from index i (a multiple of 4).
// Every device array is a 256-byte-aligned allocation with 256 bytes of
// tail padding, so the load stays inside it when some of the four indices
// are past the end (those values are not used).
__device__ __forceinline__ void load4(const int32_t *p, int32_t (&o)[4])
{
    const int4 q = __ldg(reinterpret_cast<const int4 *>(p));
    o[0] = q.x, o[1] = q.y, o[2] = q.z, o[3] = q.w;
}
__device__ __forceinline__ void load4(const float *p, float (&o)[4])
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = q.x, o[1] = q.y, o[2] = q.z, o[3] = q.w;
}
__device__ __forceinline__ void load4(const double *p, double (&o)[4])
{
    const double2 q0 = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 q1 = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = q0.x, o[1] = q0.y, o[2] = q1.x, o[3] = q1.y;
}
__device__ __forceinline__ void load4(const uint8_t *p, uint8_t (&o)[4])
{
    const uint32_t q = __ldg(reinterpret_cast<const unsigned int *>(p));
    o[0] = (uint8_t)q, o[1] = (uint8_t)(q >> 8), o[2] = (uint8_t)(q >> 16), o[3] = (uint8_t)(q >> 24);
}

// The state -> the caller's T, in the caller's node order.  Four
// consecutive nodes per thread: the internal-side arrays (permutation, home
// slot, C, Lc, phase) come in one 16-byte load each, and the four E
// gathers and T scatters are independent.
constexpr int kReadNodes = 4;
template <typename real, typename io = double>
__global__ void __launch_bounds__(256, sizeof(real) == 4 ? 6 : 4)
    k_get_temperature(StateView<real> v, io *T_out, const int32_t *node_old, int64_t n, int *err)
{
    bool bad = false;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * kReadNodes;
    for (int64_t i0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * kReadNodes; i0 < n; i0 += stride) {
        int32_t no[4], hm[4] = {0, 0, 0, 0};
        real C[4] = {}, Lc[4] = {};
        uint8_t ph[4] = {0, 0, 0, 0};
        load4(node_old + i0, no);
        if (v.home && i0 < v.n_int) load4(v.home + i0, hm);
        if (!v.is_T) {
            load4(v.C + i0, C);
            load4(v.Lc + i0, Lc);
            load4(v.ph + i0, ph);
        }
        real E[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int64_t i = i0 + u;
            E[u] = i >= n ? real(0)
                          : (i < v.n_int ? __ldg(v.Eloc + (v.home ? hm[u] : i)) : __ldg(v.Esh + (i - v.n_int)));
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            if (i0 + u >= n) break;
            const real T = v.is_T ? E[u] : temperature_of(E[u], C[u], Lc[u], ph[u], v.ranges);
            bad |= !isfinite((double)T);
            T_out[no[u]] = (io)T;
        }
    }
    if (bad && err) atomicOr(err, kErrNonFinite);
}

template <typename real>
__global__ void k_get_state(StateView<real> v, double *E_out, const int32_t *node_old, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        E_out[node_old[i]] = (double)state_E(v, i);
}

template <typename real, int NT>
__global__ void __launch_bounds__(NT) k_energy_snapshot(StateView<real> v, const real *C,
                                                        const real *Lc, const uint8_t *ph,
                                                        const real *ranges, int64_t n, double *part)
{
    double acc[2] = {0.0, 0.0};
    for (int64_t i = (int64_t)blockIdx.x * NT + threadIdx.x; i < n; i += (int64_t)gridDim.x * NT) {
        const real E = state_E(v, i);
        acc[0] += (double)E;
        acc[1] += latent_of(E, C[i], Lc[i], ph[i], ranges);
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

}  // namespace

template <typename real>
int launch_set_temperature(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, const double *T_in, const int32_t *node_old,
                           const double *dirT_int, int64_t n, void *stream)
{
    k_set_temperature<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(
        v, C, Lc, ph, ranges, T_in, node_old, dirT_int, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_set_state(StateView<real> v, const double *E_in, const int32_t *node_old, int64_t n,
                     int *err, void *stream, const int32_t *sh_ptr, const int32_t *mpos,
                     int64_t n_loc)
{
    k_set_state<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, E_in, node_old, n, err, sh_ptr,
                                                                       mpos, n_loc);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_get_temperature(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, double *T_out, const int32_t *node_old, int64_t n,
                           int *err, void *stream)
{
    k_get_temperature<real><<<grid_for((n + kReadNodes - 1) / kReadNodes, 256), 256, 0,
                                (cudaStream_t)stream>>>(v, T_out, node_old, n, err);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_set_state_f32(StateView<real> v, const float *E_in, const int32_t *node_old, int64_t n,
                         int *err, void *stream, const int32_t *sh_ptr, const int32_t *mpos,
                         int64_t n_loc)
{
    k_set_state<real, float><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, E_in, node_old, n, err,
                                                                              sh_ptr, mpos, n_loc);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_get_temperature_f32(StateView<real> v, const real *ranges, float *T_out,
                               const int32_t *node_old, int64_t n, int *err, void *stream)
{
    k_get_temperature<real, float><<<grid_for((n + kReadNodes - 1) / kReadNodes, 256), 256, 0,
                                       (cudaStream_t)stream>>>(v, T_out, node_old, n, err);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_get_state(StateView<real> v, double *E_out, const int32_t *node_old, int64_t n,
                     void *stream)
{
    k_get_state<real><<<grid_for(n, 256), 256, 0, (cudaStream_t)stream>>>(v, E_out, node_old, n);
    return (int)cudaGetLastError();
}

template <typename real>
int launch_energy_snapshot(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                           const real *ranges, int64_t n, double *part, int n_ctas, void *stream)
{
    k_energy_snapshot<real, 256><<<n_ctas, 256, 0, (cudaStream_t)stream>>>(v, C, Lc, ph, ranges, n, part);
    return (int)cudaGetLastError();
}

int launch_energy_reduce(const double *pa, int64_t na, const double *pb, int64_t nb, const double *q,
                         int64_t nq, double *out, void *stream)
{
    k_energy_reduce<<<1, kReduceThreads, 0, (cudaStream_t)stream>>>(pa, na, pb, nb, q, nq, out);
    return (int)cudaGetLastError();
}

#define FEM_INSTANTIATE(real)                                                                     \
    template int launch_set_temperature<real>(StateView<real>, const real *, const real *,        \
                                              const uint8_t *, const real *, const double *,      \
                                              const int32_t *, const double *, int64_t, void *);  \
    template int launch_set_state<real>(StateView<real>, const double *, const int32_t *, int64_t, \
                                        int *, void *, const int32_t *, const int32_t *, int64_t); \
    template int launch_get_temperature<real>(StateView<real>, const real *, const real *,        \
                                              const uint8_t *, const real *, double *,            \
                                              const int32_t *, int64_t, int *, void *);           \
    template int launch_set_state_f32<real>(StateView<real>, const float *, const int32_t *, int64_t, \
                                            int *, void *, const int32_t *, const int32_t *, int64_t); \
    template int launch_get_temperature_f32<real>(StateView<real>, const real *, float *,             \
                                                  const int32_t *, int64_t, int *, void *);            \
    template int launch_get_state<real>(StateView<real>, double *, const int32_t *, int64_t,      \
                                        void *);                                                  \
    template int launch_energy_snapshot<real>(StateView<real>, const real *, const real *,        \
                                              const uint8_t *, const real *, int64_t, double *,   \
                                              int, void *);

FEM_INSTANTIATE(float)
FEM_INSTANTIATE(double)

}  // namespace fem
