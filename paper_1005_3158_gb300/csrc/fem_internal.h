// Internal declarations shared by the host side of libfem (fem_plan.cpp,
// fem_api.cpp) and its CUDA kernels (fem_kernels.cu).  Not part of the ABI.
#pragma once

#include <cstddef>
#include <cstdint>

#ifdef __CUDACC__
#define FEM_HD __host__ __device__
#else
#define FEM_HD
#endif

namespace fem {

// Per-block header of the block-partitioned step (one CTA per block).
//   elements  [e0, e0+ne) of the block-sorted element arrays (e0 % 8 == 0)
//   faces     [f0, f0+nf) of the block-sorted face arrays   (f0 % 8 == 0)
//   interior  nodes [n0, n0+nint) of the internal numbering (owned here)
//   shared    copies [c0, c0+nsh); copy_node[c] is the internal node id
//   schedule  32-lane groups [g0, g0+ngrp]: grp[g0+g] .. grp[g0+g+1] are the
//             rounds of group g; local node l = 32 g + lane (interior first,
//             then shared copies in order)
//   slot layout in shared memory: element corner c of local element e at
//             c*ne_pad + e; face corner c of local face f at
//             4*ne_pad + c*nf_pad + f
//   weights   the block's six conductance rows are one contiguous chunk
//             w[6*e0 + k*nep + e] (nep = ne rounded up to 8)
//   rounds    [r0, r0+nrounds) of the schedule (64 bytes each); each group
//             has an even number of rounds, stored as one 32-bit word (two
//             slot indices) per lane and pair of rounds; padding entries
//             name the dummy slot 4*ne_pad + 3*nf_pad
//   chunk     the block's schedule chunk in the device stream starts at
//             32-bit word s0 = b * stride (stride: the largest chunk): a
//             header of ngrp+1 group offsets (in pairs of rounds, padded to a
//             multiple of 4 words), then the pairs (pair p, lane l at word
//             p*32 + l); one bulk copy of the whole stride moves it
struct BlockInfo {
    int32_t e0, ne, f0, nf, n0, nint, c0, nsh, g0, ngrp, ne_pad, nf_pad;
    int32_t nep, r0, nrounds, s0;
};
FEM_HD inline int32_t chunk_header_words(int32_t ngrp) { return (ngrp + 4) & ~3; }
FEM_HD inline int64_t chunk_words(const BlockInfo &b)
{
    return chunk_header_words(b.ngrp) + 16 * (int64_t)b.nrounds;
}
static_assert(sizeof(BlockInfo) == 64, "BlockInfo layout");

// Dynamic shared memory of a block-kernel CTA (16-byte aligned parts):
// [3 mbarriers, block header][conductances][schedule chunk][slots + dummy]
// [local nodes: E, partial position, phase byte], sized for the largest
// block.
constexpr size_t kSmemHdrOffset = 32;
constexpr size_t kSmemBarBytes = kSmemHdrOffset + sizeof(BlockInfo);
FEM_HD inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
FEM_HD inline size_t block_slots(const BlockInfo &b)
{
    return 4 * (size_t)b.ne_pad + 3 * (size_t)b.nf_pad + 1;  // + dummy
}
FEM_HD inline size_t block_kernel_smem(size_t nes, size_t chunk_words, size_t slots, size_t ls,
                                       size_t real_size)
{
    return kSmemBarBytes + align16(6 * nes * real_size) + align16(chunk_words * 4) +
           align16(slots * real_size) + align16(ls * (real_size + 4 + 1));
}

// Every device buffer is allocated with this many bytes after its end
// (room for 16-byte-granular bulk accesses at the end of a range).
constexpr size_t kAllocTailPad = 256;

// Bounded waits: an mbarrier wait gives up after kWaitNs nanoseconds of
// device time (or kWaitPolls polls, whichever comes first), sets the error
// flag and the step returns FEM_ETIMEOUT at the next read-back.
constexpr uint32_t kWaitPolls = 1u << 24;
constexpr unsigned long long kWaitNs = 500000000ull;
// Local nodes of one block are held in registers, kMaxLocalNodes / threads
// per thread; the planner keeps every block at or below this.
constexpr int kMaxLocalNodes = 1024;
// Bits of the device error flag (read and cleared by the fem_get_* calls).
constexpr int kErrWaitTimeout = 1;   // a bounded wait gave up
constexpr int kErrBadInput = 2;      // fem_set_state received a non-finite value
constexpr int kErrNonFinite = 4;     // a read-back temperature was non-finite
constexpr int kErrBadIndex = 8;      // checked build: an index failed its bounds check

constexpr uint8_t kDirichletBit = 0x80;  // in the per-node phase byte
constexpr int kMaxRanges = 127;
// points of one material's k(T) table; materials with tables: at most 255
constexpr int kKtMax = 16;          // distinct (Ts, Tl) pairs

// Where the nodal enthalpy of internal node i lives.  Flat variants: one
// dense array (home == null, n_int == n_nodes).  Block variant: interior
// node i at Eloc[home[i]] (its block's local array), shared node i at
// Esh[i - n_int].
template <typename real>
struct StateView {
    real *Eloc;
    real *Esh;
    const int32_t *home;
    int64_t n_int;
    // the state holds T instead of E (apparent-capacity formulation); the
    // node properties convert between the two
    bool is_T;
    const real *C, *Lc;
    const uint8_t *ph;
    const real *ranges;
#ifdef __CUDACC__
    __device__ __forceinline__ real &E(int64_t i) const
    {
        return i < n_int ? Eloc[home ? home[i] : i] : Esh[i - n_int];
    }
#endif
};

// Arguments of the block-variant kernels (device pointers).
template <typename real>
struct BlockArgs {
    const BlockInfo *blocks;
    int32_t n_blocks;
    // Per-block local node arrays, block b at [b*ls, (b+1)*ls): local node l
    // < nint is an interior node (its E lives here), nint <= l < nint+nsh a
    // shared node's copy (E mirrored by the exchange), the rest padding.
    int32_t ls;                // local-array stride (multiple of 32)
    real *Eloc;                // [n_blocks*ls]
    const real *CLloc;         // [n_blocks*ls][2] (1/C, Lc)
    const uint8_t *phloc;      // [n_blocks*ls] phase-range index | kDirichletBit
    const int32_t *posloc;     // [n_blocks*ls] shared copy: its position in P
    const real *ranges;        // [n_ranges][2] (Ts, Tl)
    // elements: block b's conductance rows at w[(6*b + k)*nes + e], k = 0..5
    // for corner pairs (0,1) (0,2) (0,3) (1,2) (1,3) (2,3): w_ab = -K^e_ab
    const real *w;
    int32_t nes;               // element stride of a block (multiple of 8)
    // faces: fa[p] = h A / 12, fg[p] = A/3 (h T_inf - q)
    const real *fa;
    const real *fg;
    // schedule chunks (see BlockInfo)
    const uint32_t *sched;
    int32_t chunk_words;       // schedule chunk stride = largest chunk (32-bit words)
    int32_t max_slots;         // largest slot count (+ dummy), a multiple of 4
    // shared-node exchange: node s owns P[sh_ptr[s] .. sh_ptr[s+1]); entry k
    // of that range is the partial of one copy, whose mirror sits at
    // Eloc[mpos[k]]
    real *P;
    const int32_t *sh_ptr;
    const int32_t *mpos;
    real *Esh;                 // [n_sh] E of the shared nodes
    const uint8_t *ph;         // [n_nodes] internal order (Dirichlet flag of shared nodes)
    int64_t n_int, n_sh;
    int64_t n_copies;          // entries of P (and Pc)
    // FP64 energy bookkeeping
    double *qcum;             // [n_blocks] cumulative heat through the Robin faces
    int *err;                 // device error flag (kErrWaitTimeout)
    // the blocks [b_first, b_first + b_count) and shared nodes [s_first,
    // s_end) one launch processes (a batch steps only its active instances);
    // per-block / per-shared-node time steps (null: the launch's dt)
    int32_t b_first, b_count;
    int64_t s_first, s_end;
    const real *blk_dt;
    const real *sh_dt;
    // temperature-dependent conductivity (instantiations with KT = true):
    // the weights are those of k = 1, element e of block b has material
    // emat[b*nes + e], whose table kt_n[m] points (kt_T, kt_k)[m*kKtMax + j]
    // gives k at the element's mean temperature
    const uint8_t *emat;
    const real *kt_T, *kt_k;
    const int32_t *kt_n;
    // apparent-capacity formulation (instantiations with LM = true): the
    // state is T; rv[b*nes + e] = rho V / 4 of the element, material m's
    // specific heat, latent heat and range (lm_c, lm_L, lm_Ts, lm_Tl)[m];
    // shared copies also write their capacity partials Pc (like P)
    const real *rv;
    const real *lm_c, *lm_L, *lm_Ts, *lm_Tl;
    real *Pc;
    // test hook (FEM_FAULT_SKIP_WEIGHT_COPY): announce the conductance copy
    // but never issue it, so that the wait for it runs out
    int32_t fault_skip_weights;
};

// Arguments of the atomic / coloured variants (device pointers).
template <typename real>
struct FlatArgs {
    real *E;
    const real *C;
    const real *Lc;
    const uint8_t *ph;
    const real *ranges;
    int64_t n_nodes;
    real *T;                  // [n_nodes] temperatures of step n
    real *R;                  // [n_nodes] residual accumulator
    const int32_t *conn;      // [4][e_stride] internal node ids (SoA)
    const real *w;            // [6][e_stride]
    int64_t n_elems, e_stride;
    const int32_t *fconn;     // [3][f_stride]
    const real *fa, *fg;
    int64_t n_faces, f_stride;
    double *qcum;             // [n_node_ctas] cumulative boundary heat
    int *err;                 // device error flag (checked build: kErrBadIndex)
    // temperature-dependent conductivity (KT instantiations): material of
    // element position p, tables as in BlockArgs
    const uint8_t *emat;
    const real *kt_T, *kt_k;
    const int32_t *kt_n;
};

// Launchers (fem_kernels.cu).  All return a cudaError_t as int.
// Block variant, one step = launch_block_kernel + launch_shared_update.
// kt: the instantiation with temperature-dependent conductivity
template <typename real>
int launch_block_kernel(const BlockArgs<real> &a, int threads, size_t smem_bytes, double dt,
                        void *stream, bool kt = false, bool lm = false, bool wg = false);
template <typename real>
int launch_shared_update(const BlockArgs<real> &a, double dt, void *stream);
// Interface faces (Eq. 8): fg[pos[f]] = g[f] * mean T of nodes sis[f][0..2]
// (internal ids), before every step's element pass.
template <typename real>
int launch_interface(StateView<real> v, const real *C, const real *Lc, const uint8_t *ph,
                     const real *ranges, real *fg, const int32_t *pos, const int32_t *sis,
                     const real *g, int64_t n, void *stream);
template <typename real>
int configure_block_kernel(int threads, size_t smem_bytes, bool kt = false, bool lm = false,
                           bool wg = false);
template <typename real>
int block_kernel_occupancy(int threads, size_t smem_bytes, int *ctas_per_sm, bool kt = false,
                           bool lm = false, bool wg = false);
// Mirrors of the shared nodes' E in the block-local arrays follow Esh
// (after the state was set from outside).
template <typename real>
int launch_mirror_copies(const BlockArgs<real> &a, void *stream);

// Flat variants, one step = temperatures, element pass (atomic adds, or one
// launch per colour with plain adds), node update with the Robin faces
// gathered through the node -> faces CSR (nf_ptr, nf_idx).
template <typename real>
int launch_flat_temperature(const FlatArgs<real> &a, void *stream);
template <typename real>
int launch_flat_elements(const FlatArgs<real> &a, bool atomic, const int64_t *color_start,
                         int n_colors, void *stream);
template <typename real>
int launch_flat_update(const FlatArgs<real> &a, const int32_t *nf_ptr, const int32_t *nf_idx,
                       int n_node_ctas, double dt, void *stream);

// Sets the calling thread's fem_last_error() message (fem_api.cpp).
void set_last_error(const char *msg);

}  // namespace fem
