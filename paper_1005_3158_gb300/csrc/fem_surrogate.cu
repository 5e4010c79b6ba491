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
// Kernels of one evaluation (nodes in 128-node tiles; x, h and m stored
// tile by tile in the tensor cores' operand layout, phi row by row):
//   k_sg_tf        T(E) and liquid fraction per node
//   k_sg_feat      the 16 input channels (two lanes per node)
//   k_sg_encode    h0 = encoder and phi_1 = P_1 h0 on tcgen05 tensor cores
//   k_sg_msg_tile  graph messages m_l on CUDA cores (FP32 sums), one CTA per
//                  tile with the phi rows of the tile and of its halo staged
//                  in shared memory (k_sg_msg: the gather form, for graphs
//                  whose tiles do not fit)
//   k_sg_layer     h_l = h_{l-1} + relu(U_l [h_{l-1}; m_l] + u_l) and the
//                  next projection (or the decoder) on tcgen05, persistent
//                  over tiles with two stages of bulk copies in flight
//   backward, loss, weight-gradient and Adam kernels for training (below).
// The message sums gather 14 neighbours per node on average: sparse work,
// kept on CUDA cores; the dense per-node layers are the contractions that go
// to the tensor cores.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "fem_device.cuh"
#include "fem_internal.h"
#include "fem_mesh_access.h"
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

// Activations with K channels stored tile by tile in the tensor-core
// operand layout: tile t (nodes 128 t .. 128 t + 127) is one contiguous
// block of 256 K bytes laid out as the core-matrix operand of fem_tc.cuh,
// so one bulk copy brings a tile into shared memory ready for the MMA.
// Pointer to the 8 channels c0..c0+7 of node i.
__device__ __forceinline__ uint16_t *tile_chunk(uint16_t *base, int64_t i, uint32_t c0, uint32_t K)
{
    return base + (i >> 7) * (128 * (int64_t)K) + (core_off((uint32_t)(i & 127), c0, K) >> 1);
}
__device__ __forceinline__ const uint16_t *tile_chunk(const uint16_t *base, int64_t i, uint32_t c0, uint32_t K)
{
    return base + (i >> 7) * (128 * (int64_t)K) + (core_off((uint32_t)(i & 127), c0, K) >> 1);
}
// Node i's row of a tile-layout activation, 8 channels per element.
struct TileRow {
    const uint16_t *base;
    int64_t i;
    uint32_t K;
    __device__ __forceinline__ uint4 operator[](int q) const
    {
        return *reinterpret_cast<const uint4 *>(tile_chunk(base, i, 8 * q, K));
    }
};

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

// Features x of every node.  Two lanes per node (sixteen nodes per warp):
// the conduction sums over the node's edges are split over the two lanes
// and combined by one shuffle; each lane writes 8 of the 16 bf16 channels.
__global__ void __launch_bounds__(256) k_sg_feat(Graph g, Acts a)
{
    const int lane = threadIdx.x & 31, sub = lane & 1;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
    const bool ok = i < g.n;
    float T = 0.f, f = 0.f, dT = 0.f, df = 0.f;
    if (ok) {
        const float2 me = a.tf[i];
        T = me.x;
        f = me.y;
        const int k1 = __ldg(g.rowptr + i + 1);
        int k = __ldg(g.rowptr + i) + sub;
        for (; k + 2 < k1; k += 4) {   // two neighbours per lane in flight
            const int j0 = __ldg(g.col + k), j1 = __ldg(g.col + k + 2);
            const float w0 = __ldg(g.w + k), w1 = __ldg(g.w + k + 2);
            const float2 o0 = a.tf[j0], o1 = a.tf[j1];
            dT += w0 * (o0.x - T);
            df += w0 * (o0.y - f);
            dT += w1 * (o1.x - T);
            df += w1 * (o1.y - f);
        }
        if (k < k1) {
            const float w0 = __ldg(g.w + k);
            const float2 o0 = a.tf[__ldg(g.col + k)];
            dT += w0 * (o0.x - T);
            df += w0 * (o0.y - f);
        }
    }
    dT += __shfl_xor_sync(0xffffffffu, dT, 1);
    df += __shfl_xor_sync(0xffffffffu, df, 1);
    if (i >= (int64_t)g.n_tiles * 128) return;
    constexpr float kInvTS = 1.f / kTS;
    float x[8];
#pragma unroll
    for (int c = 0; c < 8; c++) x[c] = 0.f;
    if (ok) {
        const float s = g.s[i];
        if (sub == 0) {
            const float C = g.C[i], Lc = g.Lc[i];
            x[0] = (T - kTC) * kInvTS;
            x[1] = f;
            x[2] = Lc / C * kInvTS;
            x[3] = kMacro * s * g.hA[i];
            x[4] = kMacro * s * (g.g[i] - g.hA[i] * T) * kInvTS;
            x[5] = kMacro * s * dT * kInvTS;
            x[6] = kMacro * s * df;
            x[7] = 1.f;
        } else if (g.Lc[i] > 0.f) {
            const int r = g.ph[i] & 0x7F;
            x[0] = (T - g.ranges[2 * r]) * kInvTS;
            x[1] = (T - g.ranges[2 * r + 1]) * kInvTS;
            x[2] = kMacro * s * g.wsum[i];
        } else {
            x[2] = kMacro * s * g.wsum[i];
        }
    }
    *reinterpret_cast<uint4 *>(tile_chunk(a.x, i, 8 * sub, 16)) =
        make_uint4(pack_bf2(x[0], x[1]), pack_bf2(x[2], x[3]), pack_bf2(x[4], x[5]), pack_bf2(x[6], x[7]));
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

// Encoder: x (from k_sg_feat) -> h0 -> phi_1 for every tile.
__global__ void __launch_bounds__(128, 4) k_sg_encode(Graph g, Acts a, const uint8_t *__restrict__ img,
                                                   const float *__restrict__ theta, Layout L,
                                                   int *err)
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
        st_row8(sA, tid, 0, 16, *reinterpret_cast<const uint4 *>(tile_chunk(a.x, i, 0, 16)));
        st_row8(sA, tid, 8, 16, *reinterpret_cast<const uint4 *>(tile_chunk(a.x, i, 8, 16)));
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
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint4 v = make_uint4(hp[4 * q], hp[4 * q + 1], hp[4 * q + 2], hp[4 * q + 3]);
            *reinterpret_cast<uint4 *>(tile_chunk(a.h[0], i, 8 * q, 64)) = v;
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

// The same messages tile by tile (the cache blocking of the paper's Section
// 4.2, applied to the graph): one CTA stages the phi rows of its 128-node
// tile and of the tile's halo (the neighbours outside it) in shared memory
// with coalesced 16-byte loads, then sums every node's messages from there
// through the edges' local columns (two lanes per node, 16 channels each).
constexpr int kMsgTileThreads = 256;
__global__ void __launch_bounds__(kMsgTileThreads) k_sg_msg_tile(Graph g, const uint16_t *__restrict__ phi,
                                                                 uint16_t *__restrict__ m_out)
{
    extern __shared__ __align__(16) uint4 sphi[];   // (128 + halo) rows x 4 chunks of 8 channels
    const int tile = blockIdx.x, tid = threadIdx.x;
    const int64_t r0 = (int64_t)tile * 128;
    const int h0 = __ldg(g.halo_ptr + tile), nh = __ldg(g.halo_ptr + tile + 1) - h0;
    const int nstage = (128 + nh) * 4;
    for (int q = tid; q < nstage; q += kMsgTileThreads) {
        const int row = q >> 2, part = q & 3;
        int64_t gr;
        if (row < 128) gr = r0 + row;
        else gr = __ldg(g.halo_idx + h0 + row - 128);
        sphi[q] = (gr < g.n) ? __ldg(reinterpret_cast<const uint4 *>(phi + gr * 32) + part)
                             : make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    const int r = tid >> 1, sub = tid & 1;
    const int64_t i = r0 + r;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; c++) acc[c] = 0.f;
    uint4 out[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
    if (i < g.n) {
        const int k1 = __ldg(g.rowptr + i + 1);
        for (int k = __ldg(g.rowptr + i); k < k1; k++) {
            const int lj = __ldg(g.lcol + k);
            const float w = __ldg(g.w + k);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint4 o = sphi[lj * 4 + 2 * sub + h];
                const uint32_t v4[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    acc[8 * h + 2 * e] = fmaf(w, bf_lo(v4[e]), acc[8 * h + 2 * e]);
                    acc[8 * h + 2 * e + 1] = fmaf(w, bf_hi(v4[e]), acc[8 * h + 2 * e + 1]);
                }
            }
        }
        const float ws = __ldg(g.wsum + i), sc = __ldg(g.s + i);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint4 mv = sphi[r * 4 + 2 * sub + h];
            const uint32_t v4[4] = {mv.x, mv.y, mv.z, mv.w};
            uint32_t q[4];
#pragma unroll
            for (int e = 0; e < 4; e++)
                q[e] = pack_bf2(sc * fmaf(-ws, bf_lo(v4[e]), acc[8 * h + 2 * e]),
                                sc * fmaf(-ws, bf_hi(v4[e]), acc[8 * h + 2 * e + 1]));
            out[h] = make_uint4(q[0], q[1], q[2], q[3]);
        }
    }
    *reinterpret_cast<uint4 *>(tile_chunk(m_out, i, 16 * sub, 32)) = out[0];
    *reinterpret_cast<uint4 *>(tile_chunk(m_out, i, 16 * sub + 8, 32)) = out[1];
}

// Graph messages of layer l: m_i = s_i sum_j W_ij (phi_j - phi_i), 32
// channels, FP32 sums of bf16 values, written as bf16; evaluated as
// s_i (sum_j W_ij phi_j - (sum_j W_ij) phi_i).  Two lanes per node (16
// channels each: two 16-byte gathers per neighbour and lane), sixteen nodes
// per warp; a node's neighbours are taken in pairs whose columns and
// weights the node's two lanes load together and share by shuffles.  A
// sparse gather with ~14 non-zeros per row: CUDA cores, many warps per SM to
// hide the gather latency.
__global__ void __launch_bounds__(256) k_sg_msg(Graph g, const uint16_t *__restrict__ phi,
                                                uint16_t *__restrict__ m_out)
{
    const int lane = threadIdx.x & 31, sub = lane & 1;
    const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
    const int64_t rows = (int64_t)g.n_tiles * 128;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; c++) acc[c] = 0.f;
    const bool ok = i < g.n;
    int k0 = 0, k1 = 0;
    if (ok) {
        k0 = __ldg(g.rowptr + i);
        k1 = __ldg(g.rowptr + i + 1);
    }
    int nch = (k1 - k0 + 1) >> 1;
#pragma unroll
    for (int o = 2; o < 32; o <<= 1) nch = max(nch, __shfl_xor_sync(0xffffffffu, nch, o));
    for (int c = 0; c < nch; c++) {
        const int kk = k0 + 2 * c + sub;
        const bool has = kk < k1;
        const int jj = has ? __ldg(g.col + kk) : 0;
        const float ww = has ? __ldg(g.w + kk) : 0.f;
        uint4 o[2][2];
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const int j = __shfl_sync(0xffffffffu, jj, (lane & ~1) | u);
            const uint4 *src = reinterpret_cast<const uint4 *>(phi + (int64_t)j * 32) + 2 * sub;
            o[u][0] = __ldg(src);
            o[u][1] = __ldg(src + 1);
        }
#pragma unroll
        for (int u = 0; u < 2; u++) {
            const float w = __shfl_sync(0xffffffffu, ww, (lane & ~1) | u);
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t v4[4] = {o[u][h].x, o[u][h].y, o[u][h].z, o[u][h].w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    acc[8 * h + 2 * e] = fmaf(w, bf_lo(v4[e]), acc[8 * h + 2 * e]);
                    acc[8 * h + 2 * e + 1] = fmaf(w, bf_hi(v4[e]), acc[8 * h + 2 * e + 1]);
                }
            }
        }
    }
    uint4 out[2] = {make_uint4(0u, 0u, 0u, 0u), make_uint4(0u, 0u, 0u, 0u)};
    if (ok) {
        const uint4 *me = reinterpret_cast<const uint4 *>(phi + i * 32) + 2 * sub;
        const float ws = __ldg(g.wsum + i), sc = __ldg(g.s + i);
#pragma unroll
        for (int h = 0; h < 2; h++) {
            const uint4 mv = __ldg(me + h);
            const uint32_t v4[4] = {mv.x, mv.y, mv.z, mv.w};
            uint32_t q[4];
#pragma unroll
            for (int e = 0; e < 4; e++)
                q[e] = pack_bf2(sc * fmaf(-ws, bf_lo(v4[e]), acc[8 * h + 2 * e]),
                                sc * fmaf(-ws, bf_hi(v4[e]), acc[8 * h + 2 * e + 1]));
            out[h] = make_uint4(q[0], q[1], q[2], q[3]);
        }
    }
    if (i < rows) {
        *reinterpret_cast<uint4 *>(tile_chunk(m_out, i, 16 * sub, 32)) = out[0];
        *reinterpret_cast<uint4 *>(tile_chunk(m_out, i, 16 * sub + 8, 32)) = out[1];
    }
}

// Shared-memory plan of the layer kernel: two stages of [h tile | m tile]
// (the A operand, filled by bulk copies), the U image and the second image.
constexpr uint32_t kLStage = 128 * 64 * 2 + 128 * 32 * 2;     // 24 KB
constexpr uint32_t kLA = 0;                                  // stage s at kLA + s * kLStage
constexpr uint32_t kLB1 = 2 * kLStage;                       // U_l image, 64 x 96
constexpr uint32_t kLB2 = kLB1 + 64 * 96 * 2;                // P_{l+1} or D1 image (<= 64 x 64)
constexpr uint32_t kLBias = kLB2 + 64 * 64 * 2;              // u | p or d1 | d2 (rounded)
constexpr uint32_t kLBar = kLBias + 192 * 4;                 // full[0], full[1], mma
constexpr uint32_t kLTmem = kLBar + 24;
constexpr uint32_t kLOk = kLTmem + 4;
constexpr uint32_t kSmemLayer = kLOk + 4 + 16;

// Thread 0 of a layer CTA: the bulk copies of one tile's h and m blocks into
// stage st, completing on that stage's barrier.
__device__ __forceinline__ void layer_issue(uint8_t *sm, uint32_t bar_full0, int st, int tile,
                                            const uint8_t *hsrc, const uint8_t *msrc)
{
    constexpr uint32_t kHB = 128 * 64 * 2, kMB = 128 * 32 * 2;
    uint8_t *dst = sm + kLA + st * kLStage;
    const uint32_t bf = bar_full0 + 8 * st;
    mbar_arrive_expect_tx(bf, kHB + kMB);
    bulk_load(smem_addr(dst), hsrc + (size_t)tile * kHB, kHB, bf);
    bulk_load(smem_addr(dst + kHB), msrc + (size_t)tile * kMB, kMB, bf);
}

// Bounded wait by thread 0 on barrier `bar`, outcome for every thread.
__device__ __forceinline__ bool cta_wait_bar(uint32_t bar, uint32_t parity, int *s_ok, int *err)
{
    return cta_wait(bar, parity, s_ok, err);
}

// Layer l (0-based) of the message passing, node-local: [h[l]; m[l]] ->
// h[l+1], then either the next layer's projection phi[l+1] or (LAST) the
// decoder and the new state.  Persistent over tiles with two stages: the
// bulk copies of tile n + 2 are in flight while tile n + 1 waits and tile
// n computes.  The new h is written in place over the stage's h tile (each
// thread rewrites only its own row) and feeds the second product.
template <bool LAST>
__global__ void __launch_bounds__(128, 3) k_sg_layer(Graph g, Acts a, const uint8_t *__restrict__ img,
                                                  const float *__restrict__ theta, Layout L, int l,
                                                  int train, int *err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sB1 = sm + kLB1, *sB2 = sm + kLB2;
    float *sBias = reinterpret_cast<float *>(sm + kLBias);
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(sm + kLTmem);
    int *sOk = reinterpret_cast<int *>(sm + kLOk);
    const uint32_t bar_full0 = smem_addr(sm + kLBar);   // stage st: bar_full0 + 8 st
    const uint32_t bar_mma = smem_addr(sm + kLBar + 16);
    const int tid = threadIdx.x;
    constexpr uint32_t N2 = LAST ? 64 : 32;
    constexpr uint32_t kHB = 128 * 64 * 2;   // bytes of an h tile
    const uint8_t *hsrc = reinterpret_cast<const uint8_t *>(a.h[l]);
    const uint8_t *msrc = reinterpret_cast<const uint8_t *>(a.m[l]);
    if (tid < 32) tc::tmem_alloc(sTmem, 128);
    if (tid == 0) {
        mbar_init(bar_full0, 1);
        mbar_init(bar_full0 + 8, 1);
        mbar_init(bar_mma, 1);
        mbar_fence_init();
        for (int st = 0; st < 2; st++) {
            const int tile = blockIdx.x + st * gridDim.x;
            if (tile < g.n_tiles) layer_issue(sm, bar_full0, st, tile, hsrc, msrc);
        }
    }
    copy_img(sB1, img + L.img_u[l], 64 * 96 * 2);
    copy_img(sB2, img + (LAST ? L.img_d1 : L.img_p[l + 1]), N2 * 64 * 2);
    if (tid < 64) sBias[tid] = theta[L.u[l] + tid];
    if (tid < (int)N2) sBias[64 + tid] = theta[(LAST ? L.d1 : L.p[l + 1]) + tid];
    if (LAST && tid < 64) sBias[128 + tid] = round_bf(theta[L.d2 + tid]);
    const float d2b = LAST ? theta[L.d2b] : 0.f;
    tc::fence_before();
    tc::fence_smem_async();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *sTmem;
    uint32_t mma_phase = 0;
    const uint32_t sb1 = smem_addr(sB1), sb2 = smem_addr(sB2);
    int it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x, it++) {
        const int st = it & 1;
        uint8_t *sAh = sm + kLA + st * kLStage, *sAm = sAh + kHB;
        if (!cta_wait_bar(bar_full0 + 8 * st, (uint32_t)((it >> 1) & 1), sOk, err)) { ok = false; break; }
        const int64_t i = (int64_t)tile * 128 + tid;
        const bool valid = i < g.n;
        if (tid == 0) {
            tc::fence_after();
            tc::mma_bf16_2seg(tbase, smem_addr(sAh), 64, smem_addr(sAm), 32, sb1, 96, 128, 64);
            tc::commit(bar_mma);
        }
        if (!cta_wait(bar_mma, mma_phase, sOk, err)) { ok = false; break; }
        mma_phase ^= 1;
        tc::fence_after();
        // r = relu(U [h; m] + u), h' = h + r (rounded to bf16), 16 columns at a time
        uint16_t *hdst = a.h[l + 1] + (int64_t)tile * (128 * 64);
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tc::ld16(tc::lane_addr(tbase, c0), v);
            uint4 hv[2] = {*reinterpret_cast<const uint4 *>(sAh + core_off(tid, c0, 64)),
                           *reinterpret_cast<const uint4 *>(sAh + core_off(tid, c0 + 8, 64))};
            uint32_t rq[8], hq[8];
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint32_t hw[4] = {hv[h].x, hv[h].y, hv[h].z, hv[h].w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    const int c = c0 + 8 * h + 2 * e;
                    const float r0 = fmaxf(v[8 * h + 2 * e] + sBias[c], 0.f);
                    const float r1 = fmaxf(v[8 * h + 2 * e + 1] + sBias[c + 1], 0.f);
                    rq[4 * h + e] = pack_bf2(r0, r1);
                    hq[4 * h + e] = valid ? pack_bf2(bf_lo(hw[e]) + r0, bf_hi(hw[e]) + r1) : 0u;
                }
            }
#pragma unroll
            for (int h = 0; h < 2; h++) {
                const uint4 nv = make_uint4(hq[4 * h], hq[4 * h + 1], hq[4 * h + 2], hq[4 * h + 3]);
                const uint32_t off = core_off(tid, c0 + 8 * h, 64);
                *reinterpret_cast<uint4 *>(sAh + off) = nv;
                *reinterpret_cast<uint4 *>(reinterpret_cast<uint8_t *>(hdst) + off) = nv;
                if (train)
                    reinterpret_cast<uint4 *>(a.r[l] + i * 64)[c0 / 8 + h] =
                        valid ? make_uint4(rq[4 * h], rq[4 * h + 1], rq[4 * h + 2], rq[4 * h + 3])
                              : make_uint4(0u, 0u, 0u, 0u);
            }
        }
        tc::fence_before();
        tc::fence_smem_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after();
            tc::mma_bf16(tbase + 64, smem_addr(sAh), sb2, 64, 128, N2, false);
            tc::commit(bar_mma);
        }
        if (!cta_wait(bar_mma, mma_phase, sOk, err)) { ok = false; break; }
        mma_phase ^= 1;
        tc::fence_after();
        if (!LAST) {
            uint32_t pp[16];
#pragma unroll
            for (int c0 = 0; c0 < 32; c0 += 16) {
                float v[16];
                tc::ld16(tc::lane_addr(tbase, 64 + c0), v);
#pragma unroll
                for (int c = 0; c < 16; c += 2)
                    pp[(c0 + c) / 2] = valid ? pack_bf2(fmaxf(v[c] + sBias[64 + c0 + c], 0.f),
                                                        fmaxf(v[c + 1] + sBias[64 + c0 + c + 1], 0.f))
                                             : 0u;
            }
            uint4 *ps = reinterpret_cast<uint4 *>(a.phi[l + 1] + i * 32);
#pragma unroll
            for (int q = 0; q < 4; q++) ps[q] = make_uint4(pp[4 * q], pp[4 * q + 1], pp[4 * q + 2], pp[4 * q + 3]);
        } else {
            // decoder: z = relu(D1 h3 + d1), y = d2 . z + d2b, E' = E + C Y_S y
            float y = d2b;
            float4 *zs = reinterpret_cast<float4 *>(a.z + i * 64);
#pragma unroll
            for (int c0 = 0; c0 < 64; c0 += 16) {
                float v[16];
                tc::ld16(tc::lane_addr(tbase, 64 + c0), v);
#pragma unroll
                for (int c = 0; c < 16; c++) {
                    v[c] = valid ? fmaxf(v[c] + sBias[64 + c0 + c], 0.f) : 0.f;
                    y = fmaf(sBias[128 + c0 + c], v[c], y);
                }
                if (train) {
#pragma unroll
                    for (int q = 0; q < 4; q++)
                        zs[c0 / 4 + q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            if (valid) {
                if (train) a.y[i] = y;
                a.E_out[i] = fmaf(g.C[i] * kYS, y, a.E_in[i]);
            }
        }
        tc::fence_before();
        __syncthreads();
        // the stage is free again: the copies of the tile two steps ahead
        if (tid == 0) {
            const int next = tile + 2 * gridDim.x;
            if (next < g.n_tiles) {
                tc::fence_smem_async();
                layer_issue(sm, bar_full0, st, next, hsrc, msrc);
            }
        }
    }
    if (!ok && tid == 0) {
        // give the copies in flight a bounded chance to land before exit
        for (int q = 0; q < 2; q++) {
            const int k = it + q;
            const int tile = blockIdx.x + k * gridDim.x;
            if (tile < g.n_tiles) mbar_wait(bar_full0 + 8 * (k & 1), (uint32_t)((k >> 1) & 1));
        }
    }
    __syncthreads();
    tc::fence_after();
    if (tid < 32) tc::tmem_free(tbase, 128);
}

// ---------------------------------------------------------------------------
// Backward (training)
// ---------------------------------------------------------------------------
//
// Weight gradients are sums over nodes, formed on the tensor cores as
// transposed products: dW^T (inputs x outputs) = sum_n [in_n; 1]^T dout_n
// with K = the tile's 128 nodes, the node inputs written transposed into a
// 128-row operand (input channels, then a row of ones whose product is the
// bias gradient, then zero rows) and the output gradients transposed into
// the B operand.  Each persistent CTA accumulates its tiles in TMEM and
// writes one partial per weight; k_sg_reduce sums the partials in CTA
// order (deterministic).

namespace {

__device__ __forceinline__ uint16_t bf_bits(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ void st_T(uint8_t *s, uint32_t row, uint32_t col, uint32_t K, uint16_t v)
{
    *reinterpret_cast<uint16_t *>(s + core_off(row, col, K)) = v;
}
// zero `bytes` (multiple of 16) of shared memory with all threads
__device__ __forceinline__ void zero_smem(uint8_t *s, uint32_t bytes)
{
    for (uint32_t o = threadIdx.x * 16; o < bytes; o += blockDim.x * 16)
        *reinterpret_cast<uint4 *>(s + o) = make_uint4(0u, 0u, 0u, 0u);
}
// rows [r0, r0 + nr) of a TMEM accumulator (this thread's lane = row), ncols
// columns -> dst[row * ncols + col]
__device__ __forceinline__ void store_acc(uint32_t tbase, uint32_t col0, uint32_t ncols, int nr,
                                          float *dst)
{
    const int row = threadIdx.x;
    for (uint32_t c0 = 0; c0 < ncols; c0 += 16) {
        float v[16];
        tc::ld16(tc::lane_addr(tbase, col0 + c0), v);
        if (row < nr)
#pragma unroll
            for (int c = 0; c < 16; c++) dst[row * ncols + c0 + c] = v[c];
    }
}
__device__ __forceinline__ float warp_sum_f(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Shared-memory plan of the backward kernels.
constexpr uint32_t kBA1 = 0;                         // 128 x 64  node-major operand (dz / dpre)
constexpr uint32_t kBB1 = kBA1 + 128 * 64 * 2;       // <= 96 x 64 weight image
constexpr uint32_t kBA2 = kBB1 + 96 * 64 * 2;        // 128 x 128 transposed inputs [in; 1]
constexpr uint32_t kBB2 = kBA2 + 128 * 128 * 2;      // 64 x 128 transposed output gradient
constexpr uint32_t kBA3 = kBB2 + 64 * 128 * 2;       // 128 x 64  du
constexpr uint32_t kBB3 = kBA3 + 128 * 64 * 2;       // 96 x 64   U^T image
constexpr uint32_t kBA4 = kBB3 + 96 * 64 * 2;        // 128 x 128 transposed [h; m; 1]
constexpr uint32_t kBB4 = kBA4 + 128 * 128 * 2;      // 64 x 128  du^T
constexpr uint32_t kBVec = kBB4 + 64 * 128 * 2;      // 64 floats (d2 rounded) + reduction space
constexpr uint32_t kBRed = kBVec + 64 * 4;           // 4 warps x 68 floats
constexpr uint32_t kBBar = kBRed + 4 * 68 * 4;
constexpr uint32_t kBTmem = kBBar + 8;
constexpr uint32_t kBOk = kBTmem + 4;
constexpr uint32_t kSmemBwd = kBOk + 4 + 16;

// TMEM columns of the backward kernels (512 allocated, one CTA per SM)
constexpr uint32_t kTdh = 0, kTacc1 = 64, kTdx = 128, kTacc2 = 256;

// Layer lu's node-local backward from dL/dh_{lu+1} (FP32, registers dh[64]):
// du = dh * (r > 0); dX = du U (tensor cores) -> dhdir = dh + dX[:, :64],
// gm_out = s dX[:, 64:]; dU^T += [h; m; 1]^T du accumulated in kTacc2.
// Writes the operands, issues both products, waits and finishes the
// epilogue.  Returns false if a wait gave up.
__device__ bool layer_back(const Graph &g, const Acts &a, const Grads &gr, float *gm_out, int lu,
                           int64_t i, bool valid, const float (&dh)[64], uint8_t *sm, uint32_t tbase,
                           uint32_t bar, uint32_t &phase, bool first, int *sOk, int *err)
{
    const int t = threadIdx.x;
    uint8_t *sA3 = sm + kBA3, *sA4 = sm + kBA4, *sB4 = sm + kBB4;
    const uint4 *rs = reinterpret_cast<const uint4 *>(a.r[lu] + i * 64);
    const TileRow hs{a.h[lu], i, 64};
    const TileRow ms{a.m[lu], i, 32};
#pragma unroll
    for (int q = 0; q < 8; q++) {
        const uint4 rv = rs[q], hv = hs[q];
        const uint32_t rw[4] = {rv.x, rv.y, rv.z, rv.w}, hw[4] = {hv.x, hv.y, hv.z, hv.w};
        uint32_t du[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int c = 8 * q + 2 * e;
            const float d0 = (valid && bf_lo(rw[e]) > 0.f) ? dh[c] : 0.f;
            const float d1 = (valid && bf_hi(rw[e]) > 0.f) ? dh[c + 1] : 0.f;
            du[e] = pack_bf2(d0, d1);
            st_T(sB4, c, t, 128, (uint16_t)(du[e] & 0xFFFF));
            st_T(sB4, c + 1, t, 128, (uint16_t)(du[e] >> 16));
            st_T(sA4, c, t, 128, (uint16_t)(hw[e] & 0xFFFF));
            st_T(sA4, c + 1, t, 128, (uint16_t)(hw[e] >> 16));
        }
        st_row8(sA3, t, 8 * q, 64, make_uint4(du[0], du[1], du[2], du[3]));
    }
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint4 mv = ms[q];
        const uint32_t mw[4] = {mv.x, mv.y, mv.z, mv.w};
#pragma unroll
        for (int e = 0; e < 4; e++) {
            const int c = 64 + 8 * q + 2 * e;
            st_T(sA4, c, t, 128, (uint16_t)(mw[e] & 0xFFFF));
            st_T(sA4, c + 1, t, 128, (uint16_t)(mw[e] >> 16));
        }
    }
    st_T(sA4, 96, t, 128, valid ? bf_bits(1.f) : (uint16_t)0);
    tc::fence_before();
    tc::fence_smem_async();
    __syncthreads();
    if (t == 0) {
        tc::fence_after();
        tc::mma_bf16(tbase + kTdx, smem_addr(sA3), smem_addr(sm + kBB3), 64, 128, 96, false);
        tc::mma_bf16(tbase + kTacc2, smem_addr(sA4), smem_addr(sB4), 128, 128, 64, !first);
        tc::commit(bar);
    }
    if (!cta_wait(bar, phase, sOk, err)) return false;
    phase ^= 1;
    tc::fence_after();
    float4 *dd = reinterpret_cast<float4 *>(gr.dhdir + i * 64);
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 16) {
        float v[16];
        tc::ld16(tc::lane_addr(tbase, kTdx + c0), v);
#pragma unroll
        for (int q = 0; q < 4; q++)
            dd[c0 / 4 + q] = valid ? make_float4(dh[c0 + 4 * q] + v[4 * q], dh[c0 + 4 * q + 1] + v[4 * q + 1],
                                                 dh[c0 + 4 * q + 2] + v[4 * q + 2],
                                                 dh[c0 + 4 * q + 3] + v[4 * q + 3])
                                   : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const float s = valid ? g.s[i] : 0.f;
    float4 *gs = reinterpret_cast<float4 *>(gm_out + i * 32);
#pragma unroll
    for (int c0 = 0; c0 < 32; c0 += 16) {
        float v[16];
        tc::ld16(tc::lane_addr(tbase, kTdx + 64 + c0), v);
#pragma unroll
        for (int q = 0; q < 4; q++)
            gs[c0 / 4 + q] = make_float4(s * v[4 * q], s * v[4 * q + 1], s * v[4 * q + 2], s * v[4 * q + 3]);
    }
    tc::fence_before();
    return true;
}

}  // namespace

// Loss and the decoder's backward pass, then layer 3's node-local backward.
//   y* = (E* - E) / (C Y_S), loss = mean (y - y*)^2, dy = 2 (y - y*) / n,
//   dd2 = sum dy z, dd2b = sum dy, dz = dy d2 (z > 0),
//   dD1^T += [h3; 1]^T dz, dh3 = dz D1.
__global__ void __launch_bounds__(128) k_sg_bwd_head(Graph g, Acts a, Grads gr, float *gm_out,
                                                     const uint8_t *__restrict__ img,
                                                     const float *__restrict__ theta, Layout L,
                                                     int *err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sA1 = sm + kBA1, *sB1 = sm + kBB1, *sA2 = sm + kBA2, *sB2 = sm + kBB2;
    float *sD2 = reinterpret_cast<float *>(sm + kBVec);
    float *sRed = reinterpret_cast<float *>(sm + kBRed);
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(sm + kBTmem);
    int *sOk = reinterpret_cast<int *>(sm + kBOk);
    const uint32_t bar = smem_addr(sm + kBBar);
    const int t = threadIdx.x;
    const int lu = kLayers - 1;
    if (t < 32) tc::tmem_alloc(sTmem, 512);
    if (t == 0) { mbar_init(bar, 1); mbar_fence_init(); }
    zero_smem(sA2, 128 * 128 * 2);
    zero_smem(sm + kBA4, 128 * 128 * 2);
    copy_img(sB1, img + L.img_d1t, 64 * 64 * 2);
    copy_img(sm + kBB3, img + L.img_ut[lu], 96 * 64 * 2);
    if (t < 64) sD2[t] = round_bf(theta[L.d2 + t]);
    tc::fence_before();
    tc::fence_smem_async();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *sTmem;
    uint32_t phase = 0;
    float acc_d2[64];
#pragma unroll
    for (int c = 0; c < 64; c++) acc_d2[c] = 0.f;
    float acc_d2b = 0.f;
    double loss = 0.0;
    bool first = true, ok = true;
    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x) {
        const int64_t i = (int64_t)tile * 128 + t;
        const bool valid = i < g.n;
        float dy = 0.f;
        if (valid) {
            const float ys = (gr.E_star[i] - a.E_in[i]) / (g.C[i] * kYS);
            const float d = a.y[i] - ys;
            loss += (double)d * (double)d;
            dy = 2.f * d * gr.inv_n;
        }
        acc_d2b += dy;
        const float4 *zs = reinterpret_cast<const float4 *>(a.z + i * 64);
        const TileRow hs{a.h[kLayers], i, 64};
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const float4 z0 = zs[2 * q], z1 = zs[2 * q + 1];
            const float zv[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
            uint32_t dz[4];
#pragma unroll
            for (int e = 0; e < 4; e++) {
                const int c = 8 * q + 2 * e;
                acc_d2[c] = fmaf(dy, zv[2 * e], acc_d2[c]);
                acc_d2[c + 1] = fmaf(dy, zv[2 * e + 1], acc_d2[c + 1]);
                const float d0 = zv[2 * e] > 0.f ? dy * sD2[c] : 0.f;
                const float d1 = zv[2 * e + 1] > 0.f ? dy * sD2[c + 1] : 0.f;
                dz[e] = pack_bf2(d0, d1);
                st_T(sB2, c, t, 128, (uint16_t)(dz[e] & 0xFFFF));
                st_T(sB2, c + 1, t, 128, (uint16_t)(dz[e] >> 16));
            }
            st_row8(sA1, t, 8 * q, 64, make_uint4(dz[0], dz[1], dz[2], dz[3]));
            const uint4 hv = hs[q];
            const uint32_t hw[4] = {hv.x, hv.y, hv.z, hv.w};
#pragma unroll
            for (int e = 0; e < 4; e++) {
                st_T(sA2, 8 * q + 2 * e, t, 128, (uint16_t)(hw[e] & 0xFFFF));
                st_T(sA2, 8 * q + 2 * e + 1, t, 128, (uint16_t)(hw[e] >> 16));
            }
        }
        st_T(sA2, 64, t, 128, valid ? bf_bits(1.f) : (uint16_t)0);
        tc::fence_smem_async();
        __syncthreads();
        if (t == 0) {
            tc::fence_after();
            tc::mma_bf16(tbase + kTdh, smem_addr(sA1), smem_addr(sB1), 64, 128, 64, false);
            tc::mma_bf16(tbase + kTacc1, smem_addr(sA2), smem_addr(sB2), 128, 128, 64, !first);
            tc::commit(bar);
        }
        if (!cta_wait(bar, phase, sOk, err)) { ok = false; break; }
        phase ^= 1;
        tc::fence_after();
        float dh[64];
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tc::ld16(tc::lane_addr(tbase, kTdh + c0), v);
#pragma unroll
            for (int c = 0; c < 16; c++) dh[c0 + c] = v[c];
        }
        if (!layer_back(g, a, gr, gm_out, lu, i, valid, dh, sm, tbase, bar, phase, first, sOk, err)) {
            ok = false;
            break;
        }
        first = false;
        __syncthreads();
    }
    // partials of this CTA
    float *part = gr.partial + (size_t)blockIdx.x * kPartFloats;
    __syncthreads();
    tc::fence_after();
    if (ok) {
        if (first) {   // no tile: zero partials
            for (int q = t; q < kPartD1; q += 128) part[kPartD1Off + q] = 0.f;
            for (int q = t; q < kPartU; q += 128) part[part_U(lu) + q] = 0.f;
        } else {
            store_acc(tbase, kTacc1, 64, 65, part + kPartD1Off);
            store_acc(tbase, kTacc2, 64, 97, part + part_U(lu));
        }
    }
    const int warp = t >> 5, lane = t & 31;
#pragma unroll
    for (int c = 0; c < 64; c++) {
        const float v = warp_sum_f(acc_d2[c]);
        if (lane == 0) sRed[warp * 68 + c] = v;
    }
    {
        const float v = warp_sum_f(acc_d2b);
        if (lane == 0) sRed[warp * 68 + 64] = v;
    }
    double lw = loss;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lw += __shfl_xor_sync(0xffffffffu, lw, o);
    __syncthreads();
    if (t < 65) part[kPartd2Off + t] = sRed[t] + sRed[68 + t] + sRed[136 + t] + sRed[204 + t];
    __syncthreads();
    double *sL = reinterpret_cast<double *>(sRed);
    if (lane == 0) sL[warp] = lw;
    __syncthreads();
    if (t == 0) gr.loss_part[blockIdx.x] = sL[0] + sL[1] + sL[2] + sL[3];
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (t < 32) tc::tmem_free(tbase, 512);
}

// Adjoint of layer l's messages: dpre_j = (phi_j > 0) sum_i W_ji (gm_i -
// gm_j) (the adjoint of m = s L phi for symmetric W, gm = s dL/dm), as bf16;
// evaluated as sum_i W_ji gm_i - (sum_i W_ji) gm_j.  Four lanes per node, 8
// channels each, neighbours in chunks of 4 shared by shuffles.
__global__ void __launch_bounds__(256) k_sg_msg_bwd(Graph g, const float *__restrict__ gm,
                                                    const uint16_t *__restrict__ phi,
                                                    uint16_t *__restrict__ dpre)
{
    const int lane = threadIdx.x & 31, sub = lane & 3;
    const int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 4;
    const int64_t rows = (int64_t)g.n_tiles * 128;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    const bool ok = j < g.n;
    int k0 = 0, k1 = 0;
    if (ok) {
        k0 = __ldg(g.rowptr + j);
        k1 = __ldg(g.rowptr + j + 1);
    }
    int nch = (k1 - k0 + 3) >> 2;
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) nch = max(nch, __shfl_xor_sync(0xffffffffu, nch, o));
    for (int c = 0; c < nch; c++) {
        const int kk = k0 + 4 * c + sub;
        const bool has = kk < k1;
        const int ii = has ? __ldg(g.col + kk) : 0;
        const float ww = has ? __ldg(g.w + kk) : 0.f;
        float4 o0[4], o1[4];
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const int q = __shfl_sync(0xffffffffu, ii, (lane & ~3) | u);
            o0[u] = __ldg(reinterpret_cast<const float4 *>(gm + (int64_t)q * 32) + 2 * sub);
            o1[u] = __ldg(reinterpret_cast<const float4 *>(gm + (int64_t)q * 32) + 2 * sub + 1);
        }
#pragma unroll
        for (int u = 0; u < 4; u++) {
            const float w = __shfl_sync(0xffffffffu, ww, (lane & ~3) | u);
            acc[0] = fmaf(w, o0[u].x, acc[0]);
            acc[1] = fmaf(w, o0[u].y, acc[1]);
            acc[2] = fmaf(w, o0[u].z, acc[2]);
            acc[3] = fmaf(w, o0[u].w, acc[3]);
            acc[4] = fmaf(w, o1[u].x, acc[4]);
            acc[5] = fmaf(w, o1[u].y, acc[5]);
            acc[6] = fmaf(w, o1[u].z, acc[6]);
            acc[7] = fmaf(w, o1[u].w, acc[7]);
        }
    }
    uint4 out = make_uint4(0u, 0u, 0u, 0u);
    if (ok) {
        const float4 m0 = __ldg(reinterpret_cast<const float4 *>(gm + j * 32) + 2 * sub);
        const float4 m1 = __ldg(reinterpret_cast<const float4 *>(gm + j * 32) + 2 * sub + 1);
        const float me[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
        const uint4 ph = __ldg(reinterpret_cast<const uint4 *>(phi + j * 32) + sub);
        const uint32_t pw[4] = {ph.x, ph.y, ph.z, ph.w};
        const float ws = __ldg(g.wsum + j);
        uint32_t q[4];
#pragma unroll
        for (int e = 0; e < 4; e++) {
            float d0 = fmaf(-ws, me[2 * e], acc[2 * e]), d1 = fmaf(-ws, me[2 * e + 1], acc[2 * e + 1]);
            if (!(bf_lo(pw[e]) > 0.f)) d0 = 0.f;
            if (!(bf_hi(pw[e]) > 0.f)) d1 = 0.f;
            q[e] = pack_bf2(d0, d1);
        }
        out = make_uint4(q[0], q[1], q[2], q[3]);
    }
    if (j < rows) reinterpret_cast<uint4 *>(dpre + j * 32)[sub] = out;
}

// Backward of layer l's projection, then layer l-1's node-local backward
// (l >= 1) or the encoder's (l == 0), from dpre (k_sg_msg_bwd):
//   dP_l^T += [h_l; 1]^T dpre;  dh_l = dhdir + dpre P_l
__global__ void __launch_bounds__(128) k_sg_bwd_mid(Graph g, Acts a, Grads gr,
                                                    const uint16_t *__restrict__ dpre, float *gm_out,
                                                    const uint8_t *__restrict__ img, Layout L, int l,
                                                    int *err)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sA1 = sm + kBA1, *sB1 = sm + kBB1, *sA2 = sm + kBA2, *sB2 = sm + kBB2;
    uint8_t *sA4 = sm + kBA4, *sB4 = sm + kBB4;
    uint32_t *sTmem = reinterpret_cast<uint32_t *>(sm + kBTmem);
    int *sOk = reinterpret_cast<int *>(sm + kBOk);
    const uint32_t bar = smem_addr(sm + kBBar);
    const int t = threadIdx.x;
    if (t < 32) tc::tmem_alloc(sTmem, 512);
    if (t == 0) { mbar_init(bar, 1); mbar_fence_init(); }
    zero_smem(sA2, 128 * 128 * 2);
    zero_smem(sA4, 128 * 128 * 2);
    copy_img(sB1, img + L.img_pt[l], 64 * 32 * 2);
    if (l >= 1) copy_img(sm + kBB3, img + L.img_ut[l - 1], 96 * 64 * 2);
    tc::fence_before();
    tc::fence_smem_async();
    __syncthreads();
    tc::fence_after();
    const uint32_t tbase = *sTmem;
    uint32_t phase = 0;
    bool first = true, ok = true;
    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x) {
        const int64_t tile0 = (int64_t)tile * 128;
        // dpre (from k_sg_msg_bwd): A operand (node rows) and transposed B
        {
            const int64_t r64 = tile0 + t;
            const uint4 *ds = reinterpret_cast<const uint4 *>(dpre + r64 * 32);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const uint4 v = ds[q];
                st_row8(sA1, t, 8 * q, 32, v);
                const uint32_t w4[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    st_T(sB2, 8 * q + 2 * e, t, 128, (uint16_t)(w4[e] & 0xFFFF));
                    st_T(sB2, 8 * q + 2 * e + 1, t, 128, (uint16_t)(w4[e] >> 16));
                }
            }
        }
        const int64_t i = tile0 + t;
        const bool valid = i < g.n;
        const TileRow hs{a.h[l], i, 64};
        uint32_t hw[32];
#pragma unroll
        for (int q = 0; q < 8; q++) {
            const uint4 hv = hs[q];
            hw[4 * q] = hv.x;
            hw[4 * q + 1] = hv.y;
            hw[4 * q + 2] = hv.z;
            hw[4 * q + 3] = hv.w;
#pragma unroll
            for (int e = 0; e < 4; e++) {
                st_T(sA2, 8 * q + 2 * e, t, 128, (uint16_t)(hw[4 * q + e] & 0xFFFF));
                st_T(sA2, 8 * q + 2 * e + 1, t, 128, (uint16_t)(hw[4 * q + e] >> 16));
            }
        }
        st_T(sA2, 64, t, 128, valid ? bf_bits(1.f) : (uint16_t)0);
        tc::fence_smem_async();
        __syncthreads();
        if (t == 0) {
            tc::fence_after();
            tc::mma_bf16(tbase + kTdh, smem_addr(sA1), smem_addr(sB1), 32, 128, 64, false);
            tc::mma_bf16(tbase + kTacc1, smem_addr(sA2), smem_addr(sB2), 128, 128, 32, !first);
            tc::commit(bar);
        }
        if (!cta_wait(bar, phase, sOk, err)) { ok = false; break; }
        phase ^= 1;
        tc::fence_after();
        float dh[64];
        const float4 *dd = reinterpret_cast<const float4 *>(gr.dhdir + i * 64);
#pragma unroll
        for (int c0 = 0; c0 < 64; c0 += 16) {
            float v[16];
            tc::ld16(tc::lane_addr(tbase, kTdh + c0), v);
#pragma unroll
            for (int q = 0; q < 4; q++) {
                const float4 b = dd[c0 / 4 + q];
                dh[c0 + 4 * q] = b.x + v[4 * q];
                dh[c0 + 4 * q + 1] = b.y + v[4 * q + 1];
                dh[c0 + 4 * q + 2] = b.z + v[4 * q + 2];
                dh[c0 + 4 * q + 3] = b.w + v[4 * q + 3];
            }
        }
        if (l >= 1) {
            if (!layer_back(g, a, gr, gm_out, l - 1, i, valid, dh, sm, tbase, bar, phase, first, sOk, err)) {
                ok = false;
                break;
            }
        } else {
            // encoder: d0 = dh0 (h0 > 0);  dW_in^T += [x; 1]^T d0
            const TileRow xs{a.x, i, 16};
#pragma unroll
            for (int q = 0; q < 2; q++) {
                const uint4 xv = xs[q];
                const uint32_t xw[4] = {xv.x, xv.y, xv.z, xv.w};
#pragma unroll
                for (int e = 0; e < 4; e++) {
                    st_T(sA4, 8 * q + 2 * e, t, 128, (uint16_t)(xw[e] & 0xFFFF));
                    st_T(sA4, 8 * q + 2 * e + 1, t, 128, (uint16_t)(xw[e] >> 16));
                }
            }
            st_T(sA4, 16, t, 128, valid ? bf_bits(1.f) : (uint16_t)0);
#pragma unroll
            for (int c = 0; c < 64; c += 2) {
                const uint32_t h2 = hw[c / 2];
                const float d0 = (valid && bf_lo(h2) > 0.f) ? dh[c] : 0.f;
                const float d1 = (valid && bf_hi(h2) > 0.f) ? dh[c + 1] : 0.f;
                const uint32_t q = pack_bf2(d0, d1);
                st_T(sB4, c, t, 128, (uint16_t)(q & 0xFFFF));
                st_T(sB4, c + 1, t, 128, (uint16_t)(q >> 16));
            }
            tc::fence_before();
            tc::fence_smem_async();
            __syncthreads();
            if (t == 0) {
                tc::fence_after();
                tc::mma_bf16(tbase + kTacc2, smem_addr(sA4), smem_addr(sB4), 128, 128, 64, !first);
                tc::commit(bar);
            }
            if (!cta_wait(bar, phase, sOk, err)) { ok = false; break; }
            phase ^= 1;
            tc::fence_after();
        }
        first = false;
        tc::fence_before();
        __syncthreads();
    }
    float *part = gr.partial + (size_t)blockIdx.x * kPartFloats;
    __syncthreads();
    tc::fence_after();
    if (ok) {
        float *p1 = part + part_P(l);
        float *p2 = l >= 1 ? part + part_U(l - 1) : part + kPartWinOff;
        const int n2 = l >= 1 ? kPartU : kPartWin;
        if (first) {
            for (int q = t; q < kPartP; q += 128) p1[q] = 0.f;
            for (int q = t; q < n2; q += 128) p2[q] = 0.f;
        } else {
            store_acc(tbase, kTacc1, 32, 65, p1);
            store_acc(tbase, kTacc2, 64, l >= 1 ? 97 : 17, p2);
        }
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (t < 32) tc::tmem_free(tbase, 512);
}

namespace {

// Where parameter q's gradient sits in a CTA's partial (see Grads).
__device__ __forceinline__ int partial_index(int q)
{
    if (q < kOffBin) { const int o = q / kNF, in = q % kNF; return kPartWinOff + in * 64 + o; }
    if (q < kLayerBase) return kPartWinOff + kNF * 64 + (q - kOffBin);
    if (q < kOffD1) {
        const int l = (q - kLayerBase) / kLayerSize;
        const int r = q - layer_P(l);
        if (r < kMSG * kHID) { const int o = r / kHID, in = r % kHID; return part_P(l) + in * kMSG + o; }
        if (r < kMSG * kHID + kMSG) return part_P(l) + kHID * kMSG + (r - kMSG * kHID);
        const int r2 = q - layer_U(l);
        if (r2 < kHID * (kHID + kMSG)) {
            const int o = r2 / (kHID + kMSG), in = r2 % (kHID + kMSG);
            return part_U(l) + in * 64 + o;
        }
        return part_U(l) + (kHID + kMSG) * 64 + (q - layer_u(l));
    }
    if (q < kOffd1) { const int o = (q - kOffD1) / kHID, in = (q - kOffD1) % kHID; return kPartD1Off + in * 64 + o; }
    if (q < kOffd2) return kPartD1Off + kHID * 64 + (q - kOffd1);
    return kPartd2Off + (q - kOffd2);   // d2 [64], then d2b
}

}  // namespace

// Sum the per-CTA partials in CTA order into the gradient of this pair
// (grad) and add it to the accumulated gradient (acc); the pair's loss (mean
// squared error) lands in *loss and is added to *loss_acc.
__global__ void k_sg_reduce(const float *__restrict__ partial, const double *__restrict__ loss_part,
                            int n_parts, float inv_n, float *__restrict__ grad, float *__restrict__ acc,
                            double *loss, double *loss_acc)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) {
        double s = 0.0;
        for (int b = 0; b < n_parts; b++) s += loss_part[b];
        *loss = s * (double)inv_n;
        *loss_acc += s * (double)inv_n;
    }
    if (q >= kNParams) return;
    const int pi = partial_index(q);
    float gsum = 0.f;
    for (int b = 0; b < n_parts; b++) gsum += partial[(size_t)b * kPartFloats + pi];
    grad[q] = gsum;
    acc[q] += gsum;
}

// One Adam step (Kingma and Ba, 2015) on the FP32 master weights with the
// mean of the accumulated gradients, g = acc / count: m = b1 m + (1-b1) g,
// v = b2 v + (1-b2) g^2, theta -= lr (m / bc1) / (sqrt(v / bc2) + eps) with
// bc1 = 1 - b1^t, bc2 = 1 - b2^t; the accumulator is cleared.
__global__ void k_sg_adam(float *__restrict__ acc, float count, float *__restrict__ theta,
                          float *__restrict__ mom, float *__restrict__ vel, AdamArgs ad)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= kNParams) return;
    const float g = __fdiv_rn(acc[q], count);
    acc[q] = 0.f;
    // every operation rounded on its own (no contraction into FMAs)
    const float m = __fadd_rn(__fmul_rn(ad.b1, mom[q]), __fmul_rn(ad.omb1, g));
    const float v = __fadd_rn(__fmul_rn(ad.b2, vel[q]), __fmul_rn(__fmul_rn(ad.omb2, g), g));
    mom[q] = m;
    vel[q] = v;
    const float mh = __fdiv_rn(m, ad.bc1), vh = __fdiv_rn(v, ad.bc2);
    theta[q] = __fsub_rn(theta[q], __fdiv_rn(__fmul_rn(ad.lr, mh), __fadd_rn(__fsqrt_rn(vh), ad.eps)));
}

// State transfer between the mesh's block layout and the surrogate order.
__global__ void k_sg_gather(StateView<float> v, const int32_t *__restrict__ int_id, int32_t n,
                            float *__restrict__ E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) E[i] = v.E(int_id[i]);
}
__global__ void k_sg_scatter(StateView<float> v, const int32_t *__restrict__ int_id, int32_t n,
                             const float *__restrict__ E)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v.E(int_id[i]) = E[i];
}

// Judge: the largest |E_a - E_b| / C_i over the nodes (the bound it puts
// on the temperature difference: dT/dE <= 1/C), as float bits in *out
// (non-negative floats order like their bit patterns).
__global__ void k_sg_judge(const float *__restrict__ Ea, const float *__restrict__ Eb, Graph g,
                           unsigned int *out)
{
    float v = 0.f;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.n; i += gridDim.x * blockDim.x)
        v = fmaxf(v, fabsf(Ea[i] - Eb[i]) / g.C[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(v));
}

}  // namespace sg
}  // namespace fem

// ===========================================================================
// Host side and C ABI
// ===========================================================================

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "fem.h"

using namespace fem;
using namespace fem::sg;

struct fem_surrogate {
    fem_mesh *mesh = nullptr;
    int device = -1, n_sm = 0;
    int fwd_per_sm = 1;               // resident encoder CTAs per SM (persistent grid)
    int layer_per_sm = 1;             // resident layer CTAs per SM
    int32_t n = 0, n_tiles = 0;
    int64_t nnz = 0;
    std::vector<int32_t> caller_of;   // surrogate position -> caller node
    double dt = 0.0;                  // plain mesh: the step the graph was built for
    std::vector<void *> bufs;
    Graph g{};
    Acts a{};
    Layout L{};
    ImgTable tab{};
    uint32_t img_bytes = 0;
    int32_t *int_id = nullptr;        // internal node of each surrogate position
    float *E0 = nullptr, *E1 = nullptr;
    float *theta = nullptr, *mom = nullptr, *vel = nullptr, *grad = nullptr, *acc = nullptr;
    int64_t n_acc = 0;                // pairs in the accumulated gradient
    uint8_t *img = nullptr;
    int *err = nullptr;
    bool train_ok = false;            // training buffers allocated
    float *dhdir = nullptr, *gm[2] = {nullptr, nullptr}, *partial = nullptr;
    uint16_t *dpre = nullptr;         // [rows][32] bf16, adjoint messages of one layer
    double *loss_part = nullptr, *loss = nullptr;   // loss[0]: last pair, loss[1]: accumulated
    int64_t adam_t = 0;
    bool have_params = false;
};

namespace {

fem_status sfail(fem_status st, const char *fmt, ...) __attribute__((format(printf, 2, 3)));
fem_status sfail(fem_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fem::set_last_error(buf);
    return st;
}
fem_status sok()
{
    fem::set_last_error("");
    return FEM_OK;
}

#define SCU(call)                                                                           \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return sfail(e_ == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA,          \
                         "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

template <typename T>
fem_status salloc(fem_surrogate *s, T **p, size_t count)
{
    void *q = nullptr;
    const size_t bytes = std::max<size_t>(count * sizeof(T), 16) + 256;
    SCU(cudaMalloc(&q, bytes));
    s->bufs.push_back(q);
    SCU(cudaMemset(q, 0, bytes));
    *p = (T *)q;
    return FEM_OK;
}

template <typename T>
fem_status supload(fem_surrogate *s, T **p, const std::vector<T> &h, size_t count)
{
    fem_status st = salloc(s, p, count);
    if (st) return st;
    if (!h.empty()) SCU(cudaMemcpy(*p, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FEM_OK;
}

void release(fem_surrogate *s)
{
    for (void *p : s->bufs) cudaFree(p);
    s->bufs.clear();
}

// Recursive coordinate bisection of the nodes idx[lo, hi) into runs whose
// lengths are multiples of 128 (the last run of the whole order excepted):
// the left part takes 128 * ceil(n / 256) nodes along the longest axis.
void rcb_nodes(const double *xyz, std::vector<int32_t> &idx, int64_t lo, int64_t hi)
{
    while (hi - lo > kTile) {
        double mn[3] = {1e300, 1e300, 1e300}, mx[3] = {-1e300, -1e300, -1e300};
        for (int64_t k = lo; k < hi; k++)
            for (int d = 0; d < 3; d++) {
                mn[d] = std::min(mn[d], xyz[3 * (size_t)idx[(size_t)k] + d]);
                mx[d] = std::max(mx[d], xyz[3 * (size_t)idx[(size_t)k] + d]);
            }
        int ax = 0;
        for (int d = 1; d < 3; d++)
            if (mx[d] - mn[d] > mx[ax] - mn[ax]) ax = d;
        const int64_t left = (int64_t)kTile * ((hi - lo + 2 * kTile - 1) / (2 * kTile));
        const int64_t mid = lo + std::min(left, hi - lo);
        std::nth_element(idx.begin() + lo, idx.begin() + mid, idx.begin() + hi, [&](int32_t p, int32_t q) {
            const double a = xyz[3 * (size_t)p + ax], b = xyz[3 * (size_t)q + ax];
            return a < b || (a == b && p < q);
        });
        if (mid >= hi) return;
        rcb_nodes(xyz, idx, lo, mid);
        lo = mid;
    }
}

}  // namespace

namespace {

// Image table and vector offsets of the parameter layout.
void build_layout(fem_surrogate *s)
{
    ImgTable &t = s->tab;
    t.n = 0;
    uint32_t bytes = 0;
    auto add = [&](uint32_t off, uint32_t sr, uint32_t sc, uint32_t rows, uint32_t cols, bool tr) {
        ImgEntry e{off, sr, sc, rows, cols, tr ? 1u : 0u, bytes, 0u};
        t.e[t.n++] = e;
        const uint32_t at = bytes;
        bytes += rows * cols * 2;
        bytes = (bytes + 127) & ~127u;
        return at;
    };
    Layout &L = s->L;
    L.img_win = add(kOffWin, kHID, kNF, kHID, kNF, false);
    for (int l = 0; l < kLayers; l++) {
        L.img_p[l] = add(layer_P(l), kMSG, kHID, kMSG, kHID, false);
        L.img_u[l] = add(layer_U(l), kHID, kHID + kMSG, kHID, kHID + kMSG, false);
        L.img_pt[l] = add(layer_P(l), kMSG, kHID, kHID, kMSG, true);
        L.img_ut[l] = add(layer_U(l), kHID, kHID + kMSG, kHID + kMSG, kHID, true);
    }
    L.img_d1 = add(kOffD1, kHID, kHID, kHID, kHID, false);
    L.img_d1t = add(kOffD1, kHID, kHID, kHID, kHID, true);
    s->img_bytes = bytes;
    L.b_in = kOffBin;
    for (int l = 0; l < kLayers; l++) {
        L.p[l] = layer_p(l);
        L.u[l] = layer_u(l);
    }
    L.d1 = kOffd1;
    L.d2 = kOffd2;
    L.d2b = kOffd2b;
}

fem_status build_graph(fem_surrogate *s, const SurrogateMeshView &v, const std::vector<double> &dt_node)
{
    const int64_t N = v.N, E = v.E;
    if (N > INT32_MAX / 2) return sfail(FEM_EINVAL, "too many nodes for the surrogate");
    // node order: recursive coordinate bisection per instance
    std::vector<int32_t> &ord = s->caller_of;
    ord.resize((size_t)N);
    std::iota(ord.begin(), ord.end(), 0);
    if (v.n_inst > 0) {
        for (int32_t k = 0; k < v.n_inst; k++) rcb_nodes(v.xyz, ord, v.inst_node[k], v.inst_node[k + 1]);
    } else {
        rcb_nodes(v.xyz, ord, 0, N);
    }
    std::vector<int32_t> pos((size_t)N);
    for (int64_t k = 0; k < N; k++) pos[(size_t)ord[(size_t)k]] = (int32_t)k;
    // node -> incident tets (caller ids)
    std::vector<int64_t> nt_ptr((size_t)N + 1, 0);
    for (int64_t e = 0; e < E; e++)
        for (int c = 0; c < 4; c++) nt_ptr[(size_t)v.tets[4 * e + c] + 1]++;
    for (int64_t i = 0; i < N; i++) nt_ptr[(size_t)i + 1] += nt_ptr[(size_t)i];
    std::vector<int32_t> nt((size_t)nt_ptr[(size_t)N]);
    {
        std::vector<int64_t> fill(nt_ptr.begin(), nt_ptr.end() - 1);
        for (int64_t e = 0; e < E; e++)
            for (int c = 0; c < 4; c++) nt[(size_t)fill[(size_t)v.tets[4 * e + c]]++] = (int32_t)e;
    }
    static const int kPairIdx[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};
    // assembled W_ij per surrogate row, columns in surrogate order, ascending
    std::vector<int32_t> rowptr((size_t)N + 1, 0), col;
    std::vector<float> w, wsum((size_t)N);
    col.reserve((size_t)N * 15);
    w.reserve((size_t)N * 15);
    std::vector<std::pair<int32_t, double>> row;
    for (int64_t k = 0; k < N; k++) {
        const int32_t i = ord[(size_t)k];
        row.clear();
        for (int64_t q = nt_ptr[(size_t)i]; q < nt_ptr[(size_t)i + 1]; q++) {
            const int64_t e = nt[(size_t)q];
            const int32_t *t = v.tets + 4 * e;
            int a = 0;
            while (t[a] != i) a++;
            for (int b = 0; b < 4; b++) {
                if (b == a) continue;
                const double wab = v.w[6 * e + kPairIdx[a][b]];
                const int32_t j = pos[(size_t)t[b]];
                bool found = false;
                for (auto &pr : row)
                    if (pr.first == j) { pr.second += wab; found = true; break; }
                if (!found) row.emplace_back(j, wab);
            }
        }
        std::sort(row.begin(), row.end());
        double ws = 0.0;
        for (auto &pr : row) {
            col.push_back(pr.first);
            const float wf = (float)pr.second;
            w.push_back(wf);
            ws += (double)wf;
        }
        wsum[(size_t)k] = (float)ws;
        rowptr[(size_t)k + 1] = (int32_t)col.size();
    }
    s->nnz = (int64_t)col.size();
    // tile blocking: each tile's neighbour rows outside the tile, and every
    // edge's column as a row of the staged block
    std::vector<int32_t> halo_ptr((size_t)s->n_tiles + 1, 0), halo_idx;
    std::vector<uint16_t> lcol(col.size());
    int32_t max_halo = 0;
    {
        std::vector<int32_t> slot((size_t)N, -1);
        for (int32_t t = 0; t < s->n_tiles; t++) {
            const int64_t r0 = (int64_t)t * kTile, r1 = std::min<int64_t>(N, r0 + kTile);
            const size_t h0 = halo_idx.size();
            for (int64_t r = r0; r < r1; r++)
                for (int32_t k = rowptr[(size_t)r]; k < rowptr[(size_t)r + 1]; k++) {
                    const int32_t j = col[(size_t)k];
                    int32_t l;
                    if (j >= r0 && j < r1) {
                        l = (int32_t)(j - r0);
                    } else {
                        if (slot[(size_t)j] < 0) {
                            slot[(size_t)j] = (int32_t)(halo_idx.size() - h0);
                            halo_idx.push_back(j);
                        }
                        l = kTile + slot[(size_t)j];
                    }
                    if (l > 65535) return sfail(FEM_EINVAL, "a tile's neighbourhood exceeds 65535 rows");
                    lcol[(size_t)k] = (uint16_t)l;
                }
            for (size_t q = h0; q < halo_idx.size(); q++) slot[(size_t)halo_idx[q]] = -1;
            halo_ptr[(size_t)t + 1] = (int32_t)halo_idx.size();
            max_halo = std::max<int32_t>(max_halo, (int32_t)(halo_idx.size() - h0));
        }
    }
    // node data in surrogate order
    const int64_t rows = (int64_t)s->n_tiles * kTile;
    std::vector<float> C((size_t)rows, 1.f), Lc((size_t)rows, 0.f), sv((size_t)rows, 0.f),
        hA((size_t)rows, 0.f), gg((size_t)rows, 0.f);
    std::vector<uint8_t> ph((size_t)rows, 0);
    std::vector<int32_t> iid((size_t)N);
    std::vector<double> hA_c((size_t)N, 0.0), g_c((size_t)N, 0.0);
    for (int64_t f = 0; f < v.F_rb; f++)
        for (int c = 0; c < 3; c++) {
            const int32_t nd = v.rb_faces[3 * f + c];
            hA_c[(size_t)nd] += 4.0 * v.rb_fa[f];   // h A / 3 = 4 (h A / 12)
            g_c[(size_t)nd] += v.rb_fg[f];
        }
    for (int64_t k = 0; k < N; k++) {
        const int32_t i = ord[(size_t)k];
        C[(size_t)k] = (float)v.C[i];
        Lc[(size_t)k] = (float)v.Lc[i];
        sv[(size_t)k] = (float)(dt_node[(size_t)i] / v.C[i]);
        hA[(size_t)k] = (float)hA_c[(size_t)i];
        gg[(size_t)k] = (float)g_c[(size_t)i];
        ph[(size_t)k] = v.rng_id[i];
        iid[(size_t)k] = v.node_new[i];
    }
    std::vector<float> rg(v.ranges, v.ranges + 2 * v.n_ranges);
    std::vector<float> rgf(rg.begin(), rg.end());
    fem_status st;
    int32_t *d_rowptr, *d_col;
    float *d_w, *d_wsum, *d_s, *d_C, *d_Lc, *d_hA, *d_g, *d_rg;
    uint8_t *d_ph;
    if ((st = supload(s, &d_rowptr, rowptr, rowptr.size()))) return st;
    if ((st = supload(s, &d_col, col, col.size()))) return st;
    if ((st = supload(s, &d_w, w, w.size()))) return st;
    if ((st = supload(s, &d_wsum, wsum, (size_t)rows))) return st;
    if ((st = supload(s, &d_s, sv, (size_t)rows))) return st;
    if ((st = supload(s, &d_C, C, (size_t)rows))) return st;
    if ((st = supload(s, &d_Lc, Lc, (size_t)rows))) return st;
    if ((st = supload(s, &d_hA, hA, (size_t)rows))) return st;
    if ((st = supload(s, &d_g, gg, (size_t)rows))) return st;
    if ((st = supload(s, &d_rg, rgf, rgf.size()))) return st;
    if ((st = supload(s, &d_ph, ph, (size_t)rows))) return st;
    if ((st = supload(s, &s->int_id, iid, (size_t)N))) return st;
    int32_t *d_hptr, *d_hidx;
    uint16_t *d_lcol;
    if ((st = supload(s, &d_hptr, halo_ptr, halo_ptr.size()))) return st;
    if ((st = supload(s, &d_hidx, halo_idx, halo_idx.size()))) return st;
    if ((st = supload(s, &d_lcol, lcol, lcol.size()))) return st;
    Graph &g = s->g;
    g.n = (int32_t)N;
    g.n_tiles = s->n_tiles;
    g.rowptr = d_rowptr;
    g.col = d_col;
    g.w = d_w;
    g.wsum = d_wsum;
    g.s = d_s;
    g.C = d_C;
    g.Lc = d_Lc;
    g.ph = d_ph;
    g.ranges = d_rg;
    g.hA = d_hA;
    g.g = d_g;
    g.halo_ptr = d_hptr;
    g.halo_idx = d_hidx;
    g.lcol = d_lcol;
    g.max_halo = max_halo;
    return FEM_OK;
}

}  // namespace

namespace {

fem_status launch_check(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return sfail(FEM_ECUDA, "%s launch failed: %s", what, cudaGetErrorString(e));
    return FEM_OK;
}

// Persistent grids: exactly the CTAs that are resident at once (a CTA
// that waits for a second wave would start its tiles after the others end).
int fwd_grid(const fem_surrogate *s) { return std::max(1, std::min(s->n_tiles, s->fwd_per_sm * s->n_sm)); }
int layer_grid(const fem_surrogate *s) { return std::max(1, std::min(s->n_tiles, s->layer_per_sm * s->n_sm)); }

// Message sums of one layer: tile-staged when a tile and its halo fit in
// shared memory, else the gather kernel.
constexpr int kMsgTileMaxRows = 3200;   // 200 KB of staged rows
void launch_msg(const fem_surrogate *s, const uint16_t *phi, uint16_t *m, cudaStream_t st)
{
    if (128 + s->g.max_halo <= kMsgTileMaxRows)
        k_sg_msg_tile<<<s->n_tiles, kMsgTileThreads, (size_t)(128 + s->g.max_halo) * 64, st>>>(s->g, phi, m);
    else
        k_sg_msg<<<(s->n_tiles * kTile * 2 + 255) / 256, 256, 0, st>>>(s->g, phi, m);
}
int bwd_grid(const fem_surrogate *s) { return std::max(1, std::min(s->n_tiles, s->n_sm)); }

// Forward pass from E_in (device, surrogate order) into E_out.
fem_status forward(fem_surrogate *s, const float *E_in, float *E_out, bool train, cudaStream_t st)
{
    Acts a = s->a;
    a.E_in = E_in;
    a.E_out = E_out;
    const int rows = s->n_tiles * kTile;
    k_sg_tf<<<(s->n + 255) / 256, 256, 0, st>>>(E_in, s->g, a.tf);
    k_sg_feat<<<(rows * 2 + 255) / 256, 256, 0, st>>>(s->g, a);
    k_sg_encode<<<fwd_grid(s), 128, kSmemFwd, st>>>(s->g, a, s->img, s->theta, s->L, s->err);
    for (int l = 0; l < kLayers; l++) {
        launch_msg(s, a.phi[l], a.m[l], st);
        if (l < kLayers - 1)
            k_sg_layer<false><<<layer_grid(s), 128, kSmemLayer, st>>>(s->g, a, s->img, s->theta, s->L, l,
                                                                  train ? 1 : 0, s->err);
        else
            k_sg_layer<true><<<layer_grid(s), 128, kSmemLayer, st>>>(s->g, a, s->img, s->theta, s->L, l,
                                                                 train ? 1 : 0, s->err);
    }
    return launch_check("surrogate forward");
}

fem_status pack(fem_surrogate *s, cudaStream_t st)
{
    k_sg_pack<<<dim3(8, s->tab.n), 256, 0, st>>>(s->theta, s->img, s->tab);
    return launch_check("parameter packing");
}

fem_status ensure_train(fem_surrogate *s)
{
    if (s->train_ok) return FEM_OK;
    const size_t rows = (size_t)s->n_tiles * kTile;
    fem_status st;
    if ((st = salloc(s, &s->dhdir, rows * 64))) return st;
    if ((st = salloc(s, &s->gm[0], rows * 32))) return st;
    if ((st = salloc(s, &s->gm[1], rows * 32))) return st;
    if ((st = salloc(s, &s->dpre, rows * 32))) return st;
    if ((st = salloc(s, &s->partial, (size_t)s->n_sm * kPartFloats))) return st;
    if ((st = salloc(s, &s->loss_part, (size_t)s->n_sm))) return st;
    if ((st = salloc(s, &s->loss, 2))) return st;
    s->train_ok = true;
    return FEM_OK;
}

fem_status check_err(fem_surrogate *s, cudaStream_t st)
{
    int flag = 0;
    SCU(cudaMemcpyAsync(&flag, s->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    SCU(cudaStreamSynchronize(st));
    if (flag) {
        SCU(cudaMemsetAsync(s->err, 0, sizeof(int), st));
        return sfail(FEM_ETIMEOUT, "a bounded tensor-core wait of the surrogate gave up");
    }
    return FEM_OK;
}

fem_status mesh_stream(fem_surrogate *s, StateView<float> *v, cudaStream_t *st)
{
    void *stream = nullptr;
    int dev = -1;
    int r = surrogate_mesh_device(s->mesh, v, &stream, &dev);
    if (r) return (fem_status)r;
    if (dev != s->device) return sfail(FEM_ESTATE, "the mesh moved to another device");
    SCU(cudaSetDevice(s->device));
    *st = (cudaStream_t)stream;
    return FEM_OK;
}

}  // namespace

extern "C" fem_status fem_surrogate_create(fem_mesh *m, double dt, fem_surrogate **out)
{
    if (!m || !out) return sfail(FEM_EINVAL, "NULL argument");
    *out = nullptr;
    SurrogateMeshView v{};
    int r = surrogate_mesh_view(m, &v);
    if (r) return (fem_status)r;
    if (v.prec != FEM_FP32 || v.variant != FEM_VARIANT_BLOCK || v.formulation != FEM_ENTHALPY)
        return sfail(FEM_EINVAL, "the surrogate needs an FP32 block-variant mesh in the enthalpy formulation");
    if (v.has_kt || v.has_dir || v.F_if > 0)
        return sfail(FEM_EINVAL, "the surrogate covers constant conductivity, Robin faces only "
                                 "(no Dirichlet nodes, no interface faces)");
    if (v.n_inst == 0 && !(dt > 0.0 && std::isfinite(dt)))
        return sfail(FEM_EINVAL, "dt must be positive and finite");
    std::vector<double> dt_node((size_t)v.N, dt);
    if (v.n_inst > 0)
        for (int32_t k = 0; k < v.n_inst; k++)
            for (int64_t i = v.inst_node[k]; i < v.inst_node[k + 1]; i++) dt_node[(size_t)i] = v.inst_dt[k];
    StateView<float> sv{};
    void *stream = nullptr;
    int dev = -1;
    if ((r = surrogate_mesh_device(m, &sv, &stream, &dev))) return (fem_status)r;
    if ((r = surrogate_mesh_view(m, &v))) return (fem_status)r;   // node_new of the uploaded plan
    fem_surrogate *s = new (std::nothrow) fem_surrogate();
    if (!s) return sfail(FEM_ENOMEM, "host allocation failed");
    s->mesh = m;
    s->device = dev;
    s->dt = dt;
    s->n = (int32_t)v.N;
    s->n_tiles = (int32_t)((v.N + kTile - 1) / kTile);
    fem_status st = FEM_OK;
    try {
        cudaSetDevice(dev);
        cudaDeviceGetAttribute(&s->n_sm, cudaDevAttrMultiProcessorCount, dev);
        build_layout(s);
        st = build_graph(s, v, dt_node);
        const size_t rows = (size_t)s->n_tiles * kTile;
        if (!st) st = salloc(s, &s->a.tf, rows);
        if (!st) st = salloc(s, &s->a.x, rows * 16);
        for (int l = 0; l <= kLayers && !st; l++) st = salloc(s, &s->a.h[l], rows * 64);
        for (int l = 0; l < kLayers && !st; l++) {
            st = salloc(s, &s->a.phi[l], rows * 32);
            if (!st) st = salloc(s, &s->a.m[l], rows * 32);
            if (!st) st = salloc(s, &s->a.r[l], rows * 64);
        }
        if (!st) st = salloc(s, &s->a.z, rows * 64);
        if (!st) st = salloc(s, &s->a.y, rows);
        if (!st) st = salloc(s, &s->E0, rows);
        if (!st) st = salloc(s, &s->E1, rows);
        if (!st) st = salloc(s, &s->theta, (size_t)kNParams);
        if (!st) st = salloc(s, &s->mom, (size_t)kNParams);
        if (!st) st = salloc(s, &s->vel, (size_t)kNParams);
        if (!st) st = salloc(s, &s->grad, (size_t)kNParams);
        if (!st) st = salloc(s, &s->acc, (size_t)kNParams);
        if (!st) st = salloc(s, &s->img, (size_t)s->img_bytes);
        if (!st) st = salloc(s, &s->err, 1);
        if (!st) {
            cudaFuncSetAttribute(k_sg_encode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemFwd);
            cudaFuncSetAttribute(k_sg_layer<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLayer);
            cudaFuncSetAttribute(k_sg_layer<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemLayer);
            cudaFuncSetAttribute(k_sg_bwd_head, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBwd);
            cudaFuncSetAttribute(k_sg_msg_tile, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kMsgTileMaxRows * 64);
            cudaFuncSetAttribute(k_sg_bwd_mid, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBwd);
            // resident forward CTAs per SM: registers and shared memory
            // (occupancy), and at most four 128-column TMEM allocations
            int regs_sm = 65536, smem_sm = 0;
            cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
            cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
            // at most four 128-column TMEM allocations per SM
            auto resident = [&](const void *fn, uint32_t dyn) {
                int occ = 4;
                cudaFuncAttributes fa{};
                if (cudaFuncGetAttributes(&fa, fn) == cudaSuccess) {
                    // registers are allocated per warp in units of 256
                    const int regs_cta = 4 * (((fa.numRegs * 32 + 255) / 256) * 256);
                    const int smem_cta = (int)(dyn + fa.sharedSizeBytes) + 1024;
                    if (regs_cta > 0) occ = std::min(occ, regs_sm / regs_cta);
                    if (smem_sm > 0) occ = std::min(occ, smem_sm / smem_cta);
                }
                return std::max(1, occ);
            };
            const int occ = resident((const void *)k_sg_encode, kSmemFwd);
            s->layer_per_sm = std::min(resident((const void *)k_sg_layer<false>, kSmemLayer),
                                       resident((const void *)k_sg_layer<true>, kSmemLayer));
            s->fwd_per_sm = std::max(1, occ);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = sfail(FEM_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
        }
    } catch (const std::bad_alloc &) {
        st = sfail(FEM_ENOMEM, "host allocation failed");
    }
    if (st) {
        release(s);
        delete s;
        return st;
    }
    *out = s;
    return sok();
}

extern "C" fem_status fem_surrogate_info(fem_surrogate *s, int64_t *n_nodes, int64_t *n_edges,
                                         int64_t *n_params)
{
    if (!s) return sfail(FEM_EINVAL, "NULL surrogate");
    if (n_nodes) *n_nodes = s->n;
    if (n_edges) *n_edges = s->nnz;
    if (n_params) *n_params = kNParams;
    return sok();
}

extern "C" fem_status fem_surrogate_order(fem_surrogate *s, int32_t *caller_of)
{
    if (!s || !caller_of) return sfail(FEM_EINVAL, "NULL argument");
    std::memcpy(caller_of, s->caller_of.data(), s->caller_of.size() * sizeof(int32_t));
    return sok();
}

extern "C" fem_status fem_surrogate_set_params(fem_surrogate *s, const float *theta, int64_t n)
{
    if (!s || !theta) return sfail(FEM_EINVAL, "NULL argument");
    if (n != kNParams) return sfail(FEM_EINVAL, "n = %lld parameters, expected %d", (long long)n, kNParams);
    for (int64_t q = 0; q < n; q++)
        if (!std::isfinite(theta[q])) return sfail(FEM_EINVAL, "non-finite parameter %lld", (long long)q);
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    SCU(cudaMemcpyAsync(s->theta, theta, (size_t)n * sizeof(float), cudaMemcpyHostToDevice, st));
    SCU(cudaMemsetAsync(s->mom, 0, (size_t)n * sizeof(float), st));
    SCU(cudaMemsetAsync(s->vel, 0, (size_t)n * sizeof(float), st));
    SCU(cudaMemsetAsync(s->acc, 0, (size_t)n * sizeof(float), st));
    s->n_acc = 0;
    if ((r = pack(s, st))) return r;
    SCU(cudaStreamSynchronize(st));
    s->adam_t = 0;
    s->have_params = true;
    return sok();
}

extern "C" fem_status fem_surrogate_get_params(fem_surrogate *s, float *theta, int64_t n)
{
    if (!s || !theta) return sfail(FEM_EINVAL, "NULL argument");
    if (n != kNParams) return sfail(FEM_EINVAL, "n = %lld parameters, expected %d", (long long)n, kNParams);
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    SCU(cudaMemcpyAsync(theta, s->theta, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, st));
    SCU(cudaStreamSynchronize(st));
    return sok();
}

extern "C" fem_status fem_surrogate_read_state(fem_surrogate *s, float *E_dev)
{
    if (!s || !E_dev) return sfail(FEM_EINVAL, "NULL argument");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    k_sg_gather<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, E_dev);
    return launch_check("state gather") ? FEM_ECUDA : sok();
}

extern "C" fem_status fem_surrogate_write_state(fem_surrogate *s, const float *E_dev)
{
    if (!s || !E_dev) return sfail(FEM_EINVAL, "NULL argument");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    k_sg_scatter<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, E_dev);
    if ((r = launch_check("state scatter"))) return r;
    r = (fem_status)surrogate_mesh_advanced(s->mesh, 0, 0.0);
    return r ? r : sok();
}

extern "C" fem_status fem_surrogate_predict(fem_surrogate *s, const float *E_in, float *E_out)
{
    if (!s || !E_in || !E_out) return sfail(FEM_EINVAL, "NULL argument");
    if (!s->have_params) return sfail(FEM_ESTATE, "no parameters (fem_surrogate_set_params)");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    r = forward(s, E_in, E_out, false, st);
    return r ? r : sok();
}

namespace {

// Forward (saving activations), loss, backward and the gradient reduction
// of one pair; the gradient is added to the accumulator.
fem_status accumulate_pair(fem_surrogate *s, const float *E_in, const float *E_star, double *loss_out,
                           cudaStream_t st)
{
    fem_status r;
    if ((r = ensure_train(s))) return r;
    if ((r = forward(s, E_in, s->E1, true, st))) return r;
    Grads gr{};
    gr.E_star = E_star;
    gr.dhdir = s->dhdir;
    gr.partial = s->partial;
    gr.loss_part = s->loss_part;
    gr.inv_n = 1.f / (float)s->n;
    Acts a = s->a;
    a.E_in = E_in;
    a.E_out = s->E1;
    const int gb = bwd_grid(s);
    k_sg_bwd_head<<<gb, 128, kSmemBwd, st>>>(s->g, a, gr, s->gm[0], s->img, s->theta, s->L, s->err);
    for (int l = kLayers - 1; l >= 0; l--) {
        const float *gin = s->gm[(kLayers - 1 - l) & 1];
        float *gout = s->gm[(kLayers - l) & 1];
        k_sg_msg_bwd<<<(s->n_tiles * kTile * 4 + 255) / 256, 256, 0, st>>>(s->g, gin, a.phi[l], s->dpre);
        k_sg_bwd_mid<<<gb, 128, kSmemBwd, st>>>(s->g, a, gr, s->dpre, gout, s->img, s->L, l, s->err);
    }
    if ((r = launch_check("surrogate backward"))) return r;
    k_sg_reduce<<<(kNParams + 255) / 256, 256, 0, st>>>(s->partial, s->loss_part, gb, 1.f / (float)s->n,
                                                        s->grad, s->acc, s->loss, s->loss + 1);
    if ((r = launch_check("gradient reduction"))) return r;
    s->n_acc += 1;
    if (loss_out) {
        SCU(cudaMemcpyAsync(loss_out, s->loss, sizeof(double), cudaMemcpyDeviceToHost, st));
        if ((r = check_err(s, st))) return r;
    }
    return FEM_OK;
}

// One Adam step of size lr with the mean of the accumulated gradients.
fem_status apply_adam(fem_surrogate *s, float lr, cudaStream_t st)
{
    AdamArgs ad{};
    const double b1 = 0.9, b2 = 0.999;
    s->adam_t += 1;
    const double t = (double)s->adam_t;
    ad.lr = lr;
    ad.b1 = (float)b1;
    ad.b2 = (float)b2;
    ad.omb1 = (float)(1.0 - b1);
    ad.omb2 = (float)(1.0 - b2);
    ad.eps = 1e-8f;
    ad.bc1 = (float)(1.0 - std::pow(b1, t));
    ad.bc2 = (float)(1.0 - std::pow(b2, t));
    k_sg_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(s->acc, (float)s->n_acc, s->theta, s->mom, s->vel, ad);
    fem_status r = launch_check("Adam step");
    if (r) return r;
    s->n_acc = 0;
    SCU(cudaMemsetAsync(s->loss + 1, 0, sizeof(double), st));
    return pack(s, st);
}

}  // namespace

extern "C" fem_status fem_surrogate_accumulate(fem_surrogate *s, const float *E_in, const float *E_star,
                                               double *loss_out)
{
    if (!s || !E_in || !E_star) return sfail(FEM_EINVAL, "NULL argument");
    if (!s->have_params) return sfail(FEM_ESTATE, "no parameters (fem_surrogate_set_params)");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    r = accumulate_pair(s, E_in, E_star, loss_out, st);
    return r ? r : sok();
}

extern "C" fem_status fem_surrogate_apply(fem_surrogate *s, float lr)
{
    if (!s) return sfail(FEM_EINVAL, "NULL surrogate");
    if (!(lr > 0.f) || !std::isfinite(lr)) return sfail(FEM_EINVAL, "lr must be positive and finite");
    if (s->n_acc == 0) return sfail(FEM_ESTATE, "no accumulated gradient (fem_surrogate_accumulate)");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    r = apply_adam(s, lr, st);
    return r ? r : sok();
}

extern "C" fem_status fem_surrogate_train_step(fem_surrogate *s, const float *E_in, const float *E_star,
                                               float lr, double *loss_out)
{
    if (!s || !E_in || !E_star) return sfail(FEM_EINVAL, "NULL argument");
    if (!s->have_params) return sfail(FEM_ESTATE, "no parameters (fem_surrogate_set_params)");
    if (!(lr >= 0.f) || !std::isfinite(lr)) return sfail(FEM_EINVAL, "lr must be >= 0 and finite");
    if (s->n_acc != 0) return sfail(FEM_ESTATE, "an accumulated gradient is pending (fem_surrogate_apply)");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    if ((r = accumulate_pair(s, E_in, E_star, loss_out, st))) return r;
    if (lr > 0.f) {
        if ((r = apply_adam(s, lr, st))) return r;
    } else {   // gradient only: drop the accumulation
        SCU(cudaMemsetAsync(s->acc, 0, (size_t)kNParams * sizeof(float), st));
        SCU(cudaMemsetAsync(s->loss + 1, 0, sizeof(double), st));
        s->n_acc = 0;
    }
    return sok();
}

extern "C" fem_status fem_surrogate_advance(fem_surrogate *s, int64_t n_macro)
{
    if (!s) return sfail(FEM_EINVAL, "NULL surrogate");
    if (n_macro < 0) return sfail(FEM_EINVAL, "n_macro must be >= 0");
    if (!s->have_params) return sfail(FEM_ESTATE, "no parameters (fem_surrogate_set_params)");
    if (n_macro == 0) return sok();
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    k_sg_gather<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, s->E0);
    float *cur = s->E0, *nxt = s->E1;
    for (int64_t k = 0; k < n_macro; k++) {
        if ((r = forward(s, cur, nxt, false, st))) return r;
        std::swap(cur, nxt);
    }
    k_sg_scatter<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, cur);
    if ((r = launch_check("state scatter"))) return r;
    r = (fem_status)surrogate_mesh_advanced(s->mesh, kMacroSteps * n_macro, s->dt);
    return r ? r : sok();
}

namespace {

// Host copy of a tile-layout activation with K channels as rows [n][K].
fem_status untile(fem_surrogate *s, const uint16_t *dev, uint32_t K, uint16_t *out)
{
    const size_t rows = (size_t)s->n_tiles * kTile;
    std::vector<uint16_t> raw(rows * K);
    SCU(cudaMemcpy(raw.data(), dev, raw.size() * 2, cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < (size_t)s->n; i++)
        for (uint32_t c = 0; c < K; c++)
            out[i * K + c] = raw[(i >> 7) * 128 * K + (core_off((uint32_t)(i & 127), c, K) >> 1)];
    return FEM_OK;
}

}  // namespace

// Test hook: host copy of an internal buffer (surrogate order, padded rows
// excluded).  which: 0 x (bf16 [n][16]), 1 h_l (bf16 [n][64], l = 0..3),
// 2 phi_l (bf16 [n][32]), 3 m_l (bf16 [n][32]), 4 r_l (bf16 [n][64]),
// 5 z (f32 [n][64]), 6 y (f32 [n]), 7 gradient (f32 [n_params]),
// 8 node data (f32 [n][5]: C, Lc, s, hA, g), 9 CSR (int32 rowptr [n+1]
// then col [nnz], then f32 w [nnz]).  Synchronises.
extern "C" fem_status fem_surrogate_debug(fem_surrogate *s, int32_t which, int32_t layer, void *out)
{
    if (!s || !out) return sfail(FEM_EINVAL, "NULL argument");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    SCU(cudaStreamSynchronize(st));
    const size_t n = (size_t)s->n;
    const bool lok = layer >= 0 && layer < kLayers;
    switch (which) {
    case 0: if ((r = untile(s, s->a.x, 16, (uint16_t *)out))) return r; break;
    case 1:
        if (layer < 0 || layer > kLayers) return sfail(FEM_EINVAL, "layer out of range");
        if ((r = untile(s, s->a.h[layer], 64, (uint16_t *)out))) return r;
        break;
    case 3:
        if (!lok) return sfail(FEM_EINVAL, "layer out of range");
        if ((r = untile(s, s->a.m[layer], 32, (uint16_t *)out))) return r;
        break;
    case 2: case 4: {
        if (!lok) return sfail(FEM_EINVAL, "layer out of range");
        const void *src = which == 2 ? (const void *)s->a.phi[layer] : (const void *)s->a.r[layer];
        SCU(cudaMemcpy(out, src, n * (which == 4 ? 64 : 32) * 2, cudaMemcpyDeviceToHost));
        break;
    }
    case 5: SCU(cudaMemcpy(out, s->a.z, n * 64 * 4, cudaMemcpyDeviceToHost)); break;
    case 6: SCU(cudaMemcpy(out, s->a.y, n * 4, cudaMemcpyDeviceToHost)); break;
    case 7: SCU(cudaMemcpy(out, s->grad, (size_t)kNParams * 4, cudaMemcpyDeviceToHost)); break;
    case 8: {
        float *o = (float *)out;
        const float *src[5] = {s->g.C, s->g.Lc, s->g.s, s->g.hA, s->g.g};
        std::vector<float> tmp(n);
        for (int k = 0; k < 5; k++) {
            SCU(cudaMemcpy(tmp.data(), src[k], n * 4, cudaMemcpyDeviceToHost));
            for (size_t i = 0; i < n; i++) o[i * 5 + k] = tmp[i];
        }
        break;
    }
    case 9: {
        int32_t *o = (int32_t *)out;
        SCU(cudaMemcpy(o, s->g.rowptr, (n + 1) * 4, cudaMemcpyDeviceToHost));
        SCU(cudaMemcpy(o + n + 1, s->g.col, (size_t)s->nnz * 4, cudaMemcpyDeviceToHost));
        SCU(cudaMemcpy(o + n + 1 + s->nnz, s->g.w, (size_t)s->nnz * 4, cudaMemcpyDeviceToHost));
        break;
    }
    default: return sfail(FEM_EINVAL, "unknown buffer %d", which);
    }
    return check_err(s, st) ? FEM_ETIMEOUT : sok();
}

extern "C" void fem_surrogate_destroy(fem_surrogate *s)
{
    if (!s) return;
    if (s->device >= 0) cudaSetDevice(s->device);
    cudaDeviceSynchronize();
    release(s);
    delete s;
}

// Surrogate stepping with the explicit solver as judge and fallback (plain
// meshes).  Every judge_every-th macro step the explicit solver takes the 16
// steps itself and the surrogate's prediction from the same state is
// compared with them; the solver's result is kept.  If the difference,
// max_i |E_sg - E_plain| / C_i (a bound on the temperature difference),
// exceeds tol_K the solver also takes the macro steps up to the next judged
// one.  stats (may be NULL): [0] macro steps by the surrogate, [1] by the
// solver (judged ones included), [2] judged steps that failed; max_err
// (may be NULL): the largest judged difference (K).  Synchronises at every
// judged step.
extern "C" fem_status fem_surrogate_solve(fem_surrogate *s, int64_t n_macro, int32_t judge_every,
                                          double tol_K, int64_t *stats, double *max_err)
{
    if (!s) return sfail(FEM_EINVAL, "NULL surrogate");
    if (n_macro < 0 || judge_every < 0) return sfail(FEM_EINVAL, "n_macro and judge_every must be >= 0");
    if (!(tol_K > 0.0)) return sfail(FEM_EINVAL, "tol_K must be positive");
    if (!s->have_params) return sfail(FEM_ESTATE, "no parameters (fem_surrogate_set_params)");
    SurrogateMeshView mv{};
    int rr = surrogate_mesh_view(s->mesh, &mv);
    if (rr) return (fem_status)rr;
    if (mv.n_inst > 0) return sfail(FEM_EINVAL, "fem_surrogate_solve steps plain meshes only");
    int64_t n_sg = 0, n_plain = 0, n_fail = 0;
    double worst = 0.0;
    // k: the next macro step; the solver takes every step before plain_until
    // and judges step next_judge; fails: consecutive failed judgements
    int64_t k = 0, plain_until = 0, next_judge = 0;
    int fails = 0;
    fem_status r = FEM_OK;
    while (k < n_macro) {
        const bool judged = judge_every > 0 && k == next_judge;
        if (!judged && k < plain_until) {
            // the solver's macro steps up to the next judged one, in one call
            // (its step graphs then cover them)
            const int64_t run = std::min(std::min(plain_until, next_judge), n_macro) - k;
            if ((r = fem_step(s->mesh, run * kMacroSteps, s->dt))) return r;
            n_plain += run;
            k += run;
        } else if (judged) {
            StateView<float> v{};
            cudaStream_t st = nullptr;
            if ((r = mesh_stream(s, &v, &st))) return r;
            k_sg_gather<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, s->E0);
            if ((r = fem_step(s->mesh, kMacroSteps, s->dt))) return r;
            n_plain++;
            if ((r = mesh_stream(s, &v, &st))) return r;
            float *Epl = s->a.y;   // scratch rows (inference does not use y)
            k_sg_gather<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, Epl);
            if ((r = forward(s, s->E0, s->E1, false, st))) return r;
            unsigned int *jb = reinterpret_cast<unsigned int *>(s->E0);   // E0 is free again
            SCU(cudaMemsetAsync(jb, 0, sizeof(unsigned int), st));
            k_sg_judge<<<std::min(4 * s->n_sm, (s->n + 255) / 256), 256, 0, st>>>(s->E1, Epl, s->g, jb);
            if ((r = launch_check("surrogate judge"))) return r;
            unsigned int bits = 0;
            SCU(cudaMemcpyAsync(&bits, jb, sizeof(bits), cudaMemcpyDeviceToHost, st));
            SCU(cudaStreamSynchronize(st));
            float e;
            std::memcpy(&e, &bits, sizeof e);
            worst = std::max(worst, (double)e);
            // a failed judgement hands the steps up to the next one to the
            // solver; each further consecutive failure doubles that span
            int64_t span = judge_every;
            if (!((double)e <= tol_K)) {
                n_fail++;
                span = (int64_t)judge_every << std::min(fails, kMaxJudgeBackoff);
                fails++;
                plain_until = k + span;
            } else {
                fails = 0;
            }
            next_judge = k + span;
            k++;
        } else {
            int64_t run = n_macro - k;
            if (judge_every > 0) run = std::min(run, next_judge - k);
            if ((r = fem_surrogate_advance(s, run))) return r;
            n_sg += run;
            k += run;
        }
    }
    if (stats) {
        stats[0] = n_sg;
        stats[1] = n_plain;
        stats[2] = n_fail;
    }
    if (max_err) *max_err = worst;
    return sok();
}

// As n_macro forward passes from the mesh's state (the state is not
// changed), timing the kernels with CUDA events on the mesh's stream:
// ms_out [5] receives the summed device milliseconds of {0: T(E), liquid
// fraction and features, 1: encoder, 2: the three message sums, 3: the
// dense parts of layers 1 and 2, 4: layer 3 with the decoder}.  Note that
// the message sums of a layer read the previous dense kernel's output, so
// in this pass they run on stale inputs (the times are what matters).
// Measurement only (one synchronisation per pass).
extern "C" fem_status fem_surrogate_profile(fem_surrogate *s, int64_t n_macro, double *ms_out)
{
    if (!s || !ms_out) return sfail(FEM_EINVAL, "NULL argument");
    if (n_macro < 0) return sfail(FEM_EINVAL, "n_macro must be >= 0");
    if (!s->have_params) return sfail(FEM_ESTATE, "no parameters (fem_surrogate_set_params)");
    StateView<float> v{};
    cudaStream_t st = nullptr;
    fem_status r = mesh_stream(s, &v, &st);
    if (r) return r;
    for (int k = 0; k < 5; k++) ms_out[k] = 0.0;
    cudaEvent_t ev[6];
    for (int k = 0; k < 6; k++) SCU(cudaEventCreate(&ev[k]));
    k_sg_gather<<<(s->n + 255) / 256, 256, 0, st>>>(v, s->int_id, s->n, s->E0);
    Acts a = s->a;
    a.E_in = s->E0;
    a.E_out = s->E1;
    const int rows = s->n_tiles * kTile;
    for (int64_t it = 0; it < n_macro && !r; it++) {
        cudaEventRecord(ev[0], st);
        k_sg_tf<<<(s->n + 255) / 256, 256, 0, st>>>(s->E0, s->g, a.tf);
        k_sg_feat<<<(rows * 2 + 255) / 256, 256, 0, st>>>(s->g, a);
        cudaEventRecord(ev[1], st);
        k_sg_encode<<<fwd_grid(s), 128, kSmemFwd, st>>>(s->g, a, s->img, s->theta, s->L, s->err);
        cudaEventRecord(ev[2], st);
        for (int l = 0; l < kLayers; l++)
            launch_msg(s, a.phi[l], a.m[l], st);
        cudaEventRecord(ev[3], st);
        for (int l = 0; l < kLayers - 1; l++)
            k_sg_layer<false><<<layer_grid(s), 128, kSmemLayer, st>>>(s->g, a, s->img, s->theta, s->L, l, 0, s->err);
        cudaEventRecord(ev[4], st);
        k_sg_layer<true><<<layer_grid(s), 128, kSmemLayer, st>>>(s->g, a, s->img, s->theta, s->L, kLayers - 1, 0,
                                                             s->err);
        cudaEventRecord(ev[5], st);
        r = launch_check("surrogate profile");
        if (cudaEventSynchronize(ev[5]) != cudaSuccess) r = sfail(FEM_ECUDA, "event synchronisation failed");
        for (int k = 0; k < 5 && !r; k++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms_out[k] += t;
        }
    }
    for (int k = 0; k < 6; k++) cudaEventDestroy(ev[k]);
    if (r) return r;
    return check_err(s, st) ? FEM_ETIMEOUT : sok();
}
