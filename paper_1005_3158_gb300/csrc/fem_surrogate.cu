// Learned mesh surrogate of the explicit enthalpy step: a message-passing
// network on the node graph of the tet mesh that advances the nodal
// enthalpy by 16 explicit steps (Eq. 14) in one evaluation, stepping over
// the explicit stability limit of Eq. 13.  The paper has no surrogate; the
// network is this library's addition, defined here and in fem.h.
//
// Network (HID = 64, MSG = 32, three message-passing layers; weights in the
// Linear convention y = W x + b; BF16 operands, FP32 accumulation):
//     h0    = relu(W_in x + b_in)                       16 -> 64
//     phi_l = relu(P_l h_{l-1} + p_l)                   64 -> 32
//     m_l,i = s_i sum_j W_ij (phi_l,j - phi_l,i)        graph message
//     h_l   = h_{l-1} + relu(U_l [h_{l-1}; m_l] + u_l)  96 -> 64
//     z     = relu(D1 h_3 + d1),  y = d2 . z + d2b      64 -> 64 -> 1
//     E'_i  = E_i + C_i Y_S y_i
// W_ij is the assembled conductance -sum_e K^e_ab of the edge (Eq. 9),
// s_i = dt / C_i; x holds the temperature T(E) (Eqs. 5, 11), the liquid
// fraction, the lumped Robin terms of Eq. 4 and the conduction change of
// one explicit step (see fem.h for the 16 channels).
//
// Kernels (one CTA of 128 threads per 128-node tile, persistent over tiles):
//   k_sg_tf        T(E) and liquid fraction per node
//   k_sg_encode    features, h0 = encoder (tcgen05), phi_1 (tcgen05)
//   k_sg_layer     message sums on CUDA cores (8 lanes per node, 4 channels
//                  per lane, FP32), the layer's update and the next layer's
//                  projection (or the decoder) on tcgen05 tensor cores
//   backward, loss, weight-gradient and Adam kernels for training (below).
// The message sums gather 14 neighbours per node on average from a graph
// with ~14 non-zeros per row: a sparse gather, kept on CUDA cores; the
// dense per-node layers are the contractions that go to the tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fem_device.cuh"
#include "fem_internal.h"
#include "fem_surrogate.h"
#include "fem_tc.cuh"

namespace fem {
namespace sg {

namespace {

using tc::core_off;

__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xFFFF0000u); }
// two floats -> packed bf16x2 (round to nearest even), lo in the low half
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi)
{
    __nv_bfloat162 t = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&t);
}
__device__ __forceinline__ float round_bf(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Bounded wait on the CTA's MMA barrier by thread 0; every thread learns
// the outcome (false: a wait gave up, the kernel stops and flags it).
__device__ __forceinline__ bool cta_wait(uint32_t bar, uint32_t parity, int *s_ok, int *err)
{
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait(bar, parity);
        *s_ok = ok ? 1 : 0;
        if (!ok) atomicOr(err, kErrWaitTimeout);
    }
    __syncthreads();
    return *s_ok != 0;
}

// Copy `bytes` (multiple of 16) of a weight image from global to shared
// memory with all threads.
__device__ __forceinline__ void copy_img(uint8_t *dst, const uint8_t *src, uint32_t bytes)
{
    for (uint32_t o = threadIdx.x * 16; o < bytes; o += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(dst + o) = __ldg(reinterpret_cast<const uint4 *>(src + o));
}

// Write 8 consecutive bf16 columns k0..k0+7 of row r of a core-matrix operand.
__device__ __forceinline__ void st_row8(uint8_t *s, uint32_t r, uint32_t k0, uint32_t K, uint4 v)
{
    *reinterpret_cast<uint4 *>(s + core_off(r, k0, K)) = v;
}

}  // namespace

// ---------------------------------------------------------------------------
// Parameter images: FP32 master vector -> bf16 core-matrix operands
// ---------------------------------------------------------------------------

// Image j of the table: operand rows x cols taken from the master matrix at
// theta[off] (rows_src x cols_src, row-major); transposed images take
// element (r, k) from (k, r).  Padding rows/columns are zero.
__global__ void k_sg_pack(const float *__restrict__ theta, uint8_t *__restrict__ img, ImgTable tab)
{
    const int j = blockIdx.y;
    if (j >= tab.n) return;
    const ImgEntry e = tab.e[j];
    const uint32_t total = e.rows * e.cols;
    for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < total; q += gridDim.x * blockDim.x) {
        const uint32_t r = q / e.cols, k = q % e.cols;
        float v = 0.f;
        if (!e.transposed) {
            if (r < e.src_rows && k < e.src_cols) v = theta[e.off + r * e.src_cols + k];
        } else {
            if (k < e.src_rows && r < e.src_cols) v = theta[e.off + k * e.src_cols + r];
        }
        __nv_bfloat16 b = __float2bfloat16_rn(v);
        *reinterpret_cast<__nv_bfloat16 *>(img + e.byte_off + core_off(r, k, e.cols)) = b;
    }
}

// ---------------------------------------------------------------------------
// Forward
// ---------------------------------------------------------------------------

// T(E) and the liquid fraction (E - C T) / Lc of every node.
__global__ void k_sg_tf(const float *__restrict__ E, Graph g, float2 *__restrict__ tf)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const float e = E[i], C = g.C[i], Lc = g.Lc[i];
    const float T = temperature_of<float>(e, C, Lc, g.ph[i], g.ranges);
    const float f = Lc > 0.f ? (e - C * T) / Lc : 0.f;
    tf[i] = make_float2(T, f);
}

// Shared-memory plan of the forward kernels (bytes, 128-byte aligned).
constexpr uint32_t kSA = 0;                               // A operand, 128 x 96 bf16
constexpr uint32_t kSB1 = kSA + 128 * 96 * 2;             // first B image (<= 64 x 96)
constexpr uint32_t kSB2 = kSB1 + 64 * 96 * 2;             // second B image (<= 64 x 64)
constexpr uint32_t kSBias = kSB2 + 64 * 64 * 2;           // biases: 64 + 64 + 64 floats
constexpr uint32_t kSBar = kSBias + 192 * 4;              // mbarrier
constexpr uint32_t kSTmem = kSBar + 8;                    // TMEM base address
constexpr uint32_t kSOk = kSTmem + 4;
constexpr uint32_t kSmemFwd = kSOk + 4 + 16;

// Encoder: x -> h0 -> phi_1 for every tile.
__global__ void __launch_bounds__(128) k_sg_encode(Graph g, Acts a, const uint8_t *__restrict__ img,
                                                   const float *__restrict__ theta, Layout L,
                                                   int train, int *err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sA = sm + kSA, *sB1 = sm + kSB1, *sB2 = sm + kSB2;
    float *sBias = reinterpret_cast<float *>(sm + kSBias);
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(sm + kSTmem);
    int *sOk = reinterpret_cast<int *>(sm + kSOk);
    const uint32_t bar = smem_addr(sm + kSBar);
    const int tid = threadIdx.x;
    if (tid < 32) tc::tmem_alloc(sTmem, 128);
    if (tid == 0) { mbar_init(bar, 1); mbar_fence_init(); }
    copy_img(sB1, img + L.img_win, 64 * 16 * 2);
    copy_img(sB2, img + L.img_p[0], 32 * 64 * 2);
    if (tid < 64) sBias[tid] = theta[L.b_in + tid];
    if (tid < 32) sBias[64 + tid] = theta[L.p[0] + tid];
    tc::fence_before();
    tc::fence_smem_async();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *sTmem;
    uint32_t phase = 0;
    const uint32_t sa = smem_addr(sA), sb1 = smem_addr(sB1), sb2 = smem_addr(sB2);
    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x) {
        const int64_t i = (int64_t)tile * 128 + tid;
        float x[16];
#pragma unroll
        for (int c = 0; c < 16; c++) x[c] = 0.f;
        if (i < g.n) {
            const float2 me = a.tf[i];
            const float T = me.x, f = me.y, C = g.C[i], Lc = g.Lc[i], s = g.s[i];
            float dT = 0.f, df = 0.f;
            for (int k = g.rowptr[i]; k < g.rowptr[i + 1]; k++) {
                const float w = g.w[k];
                const float2 o = a.tf[g.col[k]];
                dT += w * (o.x - T);
                df += w * (o.y - f);
            }
            const float Ts = g.ranges[2 * (g.ph[i] & 0x7F)], Tl = g.ranges[2 * (g.ph[i] & 0x7F) + 1];
            const bool pc = Lc > 0.f;
            x[0] = (T - kTC) / kTS;
            x[1] = f;
            x[2] = Lc / (C * kTS);
            x[3] = kMacro * s * g.hA[i];
            x[4] = kMacro * s * (g.g[i] - g.hA[i] * T) / kTS;
            x[5] = kMacro * s * dT / kTS;
            x[6] = kMacro * s * df;
            x[7] = 1.f;
            x[8] = pc ? (T - Ts) / kTS : 0.f;
            x[9] = pc ? (T - Tl) / kTS : 0.f;
            x[10] = kMacro * s * g.wsum[i];
        }
        uint4 q0 = make_uint4(pack_bf2(x[0], x[1]), pack_bf2(x[2], x[3]), pack_bf2(x[4], x[5]),
                              pack_bf2(x[6], x[7]));
        uint4 q1 = make_uint4(pack_bf2(x[8], x[9]), pack_bf2(x[10], x[11]), pack_bf2(x[12], x[13]),
                              pack_bf2(x[14], x[15]));
        st_row8(sA, tid, 0, 16, q0);
        st_row8(sA, tid, 8, 16, q1);
        if (train) {
            uint4 *xs = reinterpret_cast<uint4 *>(a.x + (size_t)i * 16);
            xs[0] = q0;
            xs[1] = q1;
        }
        tc::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            tc::mma_bf16(tbase, sa, sb1, 16, 128, 64, false);
            tc::commit(bar);
        }
        if (!cta_wait(bar, phase, sOk, err)) break;
        phase ^= 1;
        tc::fence_after();
        // h0 = relu(acc + b_in): this thread's row
        uint32_t hp[32];
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tc::ld16(tc::lane_addr(tbase, c0), v);
#pragma unroll
            for (int c = 0; c < 16; c += 2)
                hp[(c0 + c) / 2] = pack_bf2(fmaxf(v[c] + sBias[c0 + c], 0.f),
                                            fmaxf(v[c + 1] + sBias[c0 + c + 1], 0.f));
        }
        if (i >= g.n) {
#pragma unroll
            for (int c = 0; c < 32; c++) hp[c] = 0u;
        }
        uint4 *hs = reinterpret_cast<uint4 *>(a.h[0] + (size_t)i * 64);
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint4 v = make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
            hs[q] = v;
            st_row8(sA, tid, 8 * q, 64, v);
        }
        tc::fence_before();
        tc::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            tc::mma_bf16(tbase + 64, sa, sb2, 64, 128, 32, false);
            tc::commit(bar);
        }
        if (!cta_wait(bar, phase, sOk, err)) break;
        phase ^= 1;
        tc::fence_after();
        uint32_t pp[16];
#pragma unroll
        for (int c0 = 0; c0 < 32; c0 += 16) {
            float v[16];
            tc::ld16(tc::lane_addr(tbase, 64 + c0), v);
#pragma unroll
            for (int c = 0; c < 16; c += 2)
                pp[(c0 + c) / 2] = pack_bf2(fmaxf(v[c] + sBias[64 + c0 + c], 0.f),
                                            fmaxf(v[c + 1] + sBias[64 + c0 + c + 1], 0.f));
        }
        if (i >= g.n) {
#pragma unroll
            for (int c = 0; c < 16; c++) pp[c] = 0u;
        }
        uint4 *ps = reinterpret_cast<uint4 *>(a.phi[0] + (size_t)i * 32);
#pragma unroll
        for (int q = 0; q < 4; q++) ps[q] = make_uint4(pp[4 * q], pp[4 * q + 1], pp[4 * q + 2], pp[4 * q + 3]);
        tc::fence_before();
        __syncthreads();
    }
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_free(tbase, 128);
}
