// Internal declarations of the learned surrogate (fem_surrogate.cu): sizes,
// parameter layout and the device argument structs.  Not part of the ABI.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#define SG_HD __host__ __device__
#else
#define SG_HD
#endif

namespace fem {
namespace sg {

constexpr int kNF = 16, kHID = 64, kMSG = 32, kLayers = 3, kTile = 128;
constexpr float kTC = 600.f, kTS = 300.f, kYS = 10.f, kMacro = 16.f;
constexpr int kMacroSteps = 16;
// Hybrid solve: after f consecutive failed judgements the solver takes the
// next judge_every * 2^min(f - 1, kMaxJudgeBackoff) macro steps.
constexpr int kMaxJudgeBackoff = 6;

// Flat FP32 parameter vector (the Linear convention y = W x + b):
//   W_in [64][16], b_in [64],
//   per layer l = 1..3: P_l [32][64], p_l [32], U_l [64][96], u_l [64],
//   D1 [64][64], d1 [64], d2 [64], d2b [1].
constexpr int kOffWin = 0, kOffBin = kOffWin + kHID * kNF;
constexpr int kLayerBase = kOffBin + kHID;
constexpr int kLayerSize = kMSG * kHID + kMSG + kHID * (kHID + kMSG) + kHID;
SG_HD constexpr int layer_P(int l) { return kLayerBase + l * kLayerSize; }          // l = 0..2
SG_HD constexpr int layer_p(int l) { return layer_P(l) + kMSG * kHID; }
SG_HD constexpr int layer_U(int l) { return layer_p(l) + kMSG; }
SG_HD constexpr int layer_u(int l) { return layer_U(l) + kHID * (kHID + kMSG); }
constexpr int kOffD1 = kLayerBase + kLayers * kLayerSize;
constexpr int kOffd1 = kOffD1 + kHID * kHID;
constexpr int kOffd2 = kOffd1 + kHID;
constexpr int kOffd2b = kOffd2 + kHID;
constexpr int kNParams = kOffd2b + 1;
static_assert(kNParams == 30177, "parameter count");

// One bf16 operand image (core-matrix layout, see fem_tc.cuh) built from a
// master matrix of src_rows x src_cols at theta[off]: rows x cols, possibly
// transposed.
struct ImgEntry {
    uint32_t off, src_rows, src_cols, rows, cols, transposed, byte_off, pad;
};
constexpr int kMaxImg = 16;
struct ImgTable {
    ImgEntry e[kMaxImg];
    int n;
};

// Byte offsets of the images and element offsets of the vectors the
// kernels read.
struct Layout {
    uint32_t img_win;            // W_in            64 x 16
    uint32_t img_p[kLayers];     // P_l             32 x 64
    uint32_t img_u[kLayers];     // U_l             64 x 96
    uint32_t img_d1;             // D1              64 x 64
    uint32_t img_pt[kLayers];    // P_l^T           64 x 32
    uint32_t img_ut[kLayers];    // U_l^T           96 x 64
    uint32_t img_d1t;            // D1^T            64 x 64
    int32_t b_in, p[kLayers], u[kLayers], d1, d2, d2b;
};

// The surrogate's graph and node data (device pointers, surrogate order).
struct Graph {
    int32_t n;          // nodes
    int32_t n_tiles;    // ceil(n / 128); per-node arrays hold n_tiles * 128 rows
    const int32_t *rowptr, *col;
    const float *w;     // W_ij, the assembled conductance of the edge (W/K)
    const float *wsum;  // sum_j W_ij
    const float *s;     // dt / C_i
    const float *C, *Lc;
    const uint8_t *ph;  // phase-change range index (low 7 bits)
    const float *ranges;
    const float *hA, *g;  // lumped Robin terms sum h A / 3, sum A (h T_inf - q) / 3
    // tile blocking of the message sums: the rows of tile t's neighbours
    // outside the tile are halo_idx[halo_ptr[t] .. halo_ptr[t + 1]); lcol[k]
    // is edge k's column as a row of the staged block (tile rows 0..127,
    // then the halo rows)
    const int32_t *halo_ptr, *halo_idx;
    const uint16_t *lcol;
    int32_t max_halo;
};

// Activations (surrogate order, n_tiles * 128 rows each, bf16 as uint16).
struct Acts {
    float2 *tf;                 // T, liquid fraction
    uint16_t *x;                // [rows][16]   (training)
    uint16_t *h[kLayers + 1];   // [rows][64]
    uint16_t *phi[kLayers];     // [rows][32]
    uint16_t *m[kLayers];       // [rows][32]   (training)
    uint16_t *r[kLayers];       // [rows][64]   (training)
    float *z;                   // [rows][64]   (training)
    float *y;                   // [rows]
    const float *E_in;          // [rows]
    float *E_out;               // [rows]
};

// Backward buffers.
struct Grads {
    const float *E_star;        // target state after 16 steps
    float *dhdir;               // [rows][64] FP32: dL/dh through the residual and U
    float *gm;                  // [rows][32] FP32: s_i dL/dm_i
    float *partial;             // per CTA: weight-gradient partials (kPartialFloats each)
    double *loss_part;          // per CTA: sum of squared errors
    float inv_n;                // 1 / number of nodes
};
// Weight-gradient partial of one CTA: transposed gradients, rows = input
// channel (+ one bias row), columns = output channel.
//   U_l^T: 97 x 64 per layer, P_l^T: 65 x 32 per layer, D1^T: 65 x 64,
//   W_in^T: 17 x 64, d2: 64, d2b: 1.
constexpr int kPartU = 97 * 64, kPartP = 65 * 32, kPartD1 = 65 * 64, kPartWin = 17 * 64;
SG_HD constexpr int part_U(int l) { return l * kPartU; }
SG_HD constexpr int part_P(int l) { return kLayers * kPartU + l * kPartP; }
constexpr int kPartD1Off = kLayers * (kPartU + kPartP);
constexpr int kPartWinOff = kPartD1Off + kPartD1;
constexpr int kPartd2Off = kPartWinOff + kPartWin;
constexpr int kPartFloats = kPartd2Off + 64 + 1 + 3;   // padded to a multiple of 4

// Adam hyper-parameters of one step (omb1 = 1 - b1, omb2 = 1 - b2,
// bc1 = 1 - b1^t, bc2 = 1 - b2^t, each rounded once from FP64).
struct AdamArgs {
    float lr, b1, b2, omb1, omb2, eps, bc1, bc2, inv_n;
};

}  // namespace sg
}  // namespace fem
