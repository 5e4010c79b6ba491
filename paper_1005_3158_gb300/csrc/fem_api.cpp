// C ABI of libfem (include/fem.h): argument validation, set-up of the
// stored element conductances and lumped capacities (Section 3), plan and
// device-memory management, and the step driver.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "fem.h"
#include "fem_internal.h"
#include "fem_io.h"
#include "fem_mesh_access.h"
#include "fem_plan.h"

using namespace fem;

namespace {

thread_local std::string g_err;

fem_status fail(fem_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return st;
}

fem_status ok()
{
    g_err.clear();
    return FEM_OK;
}

// ---------------------------------------------------------------------------
// Device allocations (with an allocation-failure injection hook for tests:
// FEM_FAULT_ALLOC_AFTER=k makes every device allocation after the k-th of
// one mesh upload fail; the count restarts with each upload)
// ---------------------------------------------------------------------------
long g_alloc_count = 0;

// false when the test hook says this allocation must fail
bool alloc_allowed()
{
    const char *env = getenv("FEM_FAULT_ALLOC_AFTER");
    if (env && *env && g_alloc_count >= atol(env)) return false;
    g_alloc_count++;
    return true;
}

struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

void fem::set_last_error(const char *msg) { g_err = msg ? msg : ""; }

struct fem_mesh {
    // ---- caller-order host data
    int64_t N = 0, E = 0, F = 0;
    std::vector<double> xyz;
    std::vector<int32_t> tets, mat;
    std::vector<double> vol;          // |V|
    NodeElems adj;
    std::vector<int32_t> rank;        // node priority (RCM position or identity)
    int64_t bw_input = 0, bw_rank = 0;
    fem_precision prec = FEM_FP64;
    int reorder = 0;
    fem_options opt{};
    // materials
    bool have_mat = false;
    std::vector<double> w;            // [E][6] conductances
    std::vector<double> Cn, mn, Lcn;  // lumped per node
    std::vector<uint8_t> rng_id;      // phase-range index per node
    std::vector<double> ranges;       // [nr][2]
    int32_t n_mat = 0;
    std::vector<double> mat_k;        // constant conductivity per material
    std::vector<fem_material> mats;   // the material table (apparent capacity)
    // temperature-dependent conductivity: per material a table of (T, k)
    // points (empty: constant k); has_kt when any table is set
    std::vector<std::vector<double>> kt_T, kt_k;
    bool has_kt = false;
    // boundary: Robin faces (fem_set_boundary) and interface faces
    // (fem_set_interface, Eq. 8), kept apart and combined into faces/fa/fg
    // (Robin first) for the plan, the uploads and the stable step
    std::vector<int32_t> rb_faces;
    std::vector<double> rb_fa, rb_fg;
    int64_t F_rb = 0;
    std::vector<int32_t> if_faces;    // [F_if][3], side A then side B
    std::vector<double> if_fa, if_g;  // h_i A / 12, h_i A / 3
    std::vector<int64_t> if_sister;   // index into the interface list
    std::vector<int32_t> if_sister32; // fem_plan_array view
    int64_t F_if = 0;
    std::vector<int32_t> faces;
    std::vector<double> fa, fg;       // h A / 12, A/3 (h T_inf - q); fg = 0 on interface faces
    // Dirichlet
    std::vector<uint8_t> is_dir;
    std::vector<double> dir_T;        // caller order (valid where is_dir)
    // ---- plan
    bool plan_ok = false;
    BlockPlan bp;
    FlatPlan fp;
    std::vector<int32_t> nf_ptr, nf_idx;  // flat: node -> faces (internal ids)
    std::vector<int32_t> blocks_flat;     // fem_plan_array view of bp.blocks
    // ---- device
    bool dev_ok = false;
    int device = -1;
    cudaStream_t stream = nullptr;
    std::vector<DevBuf> bufs;
    // device memory from the caller's allocator (fem_set_allocator), else cudaMalloc
    fem_alloc_fn alloc_fn = nullptr;
    fem_free_fn free_fn = nullptr;
    void *alloc_ctx = nullptr;
    size_t dev_bytes = 0;
    size_t smem_bytes = 0;
    bool wg = false;                           // block kernel reads the conductances from L2
    int threads = 256;
    int32_t chunk_words = 0, max_slots = 0, ctas_per_sm = 0;
    int n_node_ctas = 0;
    // device pointers
    void *dE = nullptr, *dC = nullptr, *dLc = nullptr, *dRanges = nullptr, *dW = nullptr,
         *dFa = nullptr, *dFg = nullptr, *dP = nullptr, *dT = nullptr, *dR = nullptr,
         *dEloc = nullptr, *dCLloc = nullptr, *dEsh = nullptr;
    uint8_t *dPhloc = nullptr;
    int32_t *dPosloc = nullptr, *dHome = nullptr, *dMpos = nullptr;
    int32_t ls = 0, nes = 0;
    uint8_t *dPh = nullptr;
    BlockInfo *dBlocks = nullptr;
    int32_t *dShPtr = nullptr,
            *dNodeOld = nullptr, *dConn = nullptr, *dFconn = nullptr, *dNfPtr = nullptr,
            *dNfIdx = nullptr;
    uint32_t *dSched = nullptr;
    int32_t *dIfPos = nullptr, *dIfSis = nullptr;   // interface: face position, sister nodes
    void *dIfG = nullptr;
    uint8_t *dEmat = nullptr;                      // k(T), apparent capacity: material per element
    void *dRv = nullptr, *dLmC = nullptr, *dLmL = nullptr, *dLmTs = nullptr, *dLmTl = nullptr,
         *dPc = nullptr;                           // apparent capacity (see BlockArgs)
    void *dKtT = nullptr, *dKtK = nullptr;         // k(T) tables [n_mat][kKtMax]
    int32_t *dKtN = nullptr;
    double *dEpart = nullptr, *dQcum = nullptr, *dIo = nullptr,
           *dDirT = nullptr, *dOut = nullptr;
    int *dErr = nullptr;
    // ---- state
    enum { ST_NONE, ST_PENDING_T, ST_PENDING_E, ST_DEVICE } state = ST_NONE;
    std::vector<double> pending;      // T0 or E (caller order)
    int64_t step = 0;
    double time = 0.0;
    double U0 = 0.0;
    double q_carry = 0.0;             // boundary heat of device buffers already released
    // energy balance check (fem_get_energy): the account is exact from
    // fem_set_temperature on, until a state is uploaded (fem_set_state*);
    // acct_steps counts the steps taken since the account began
    bool acct_exact = false;
    int64_t acct_steps = 0;
    double acct_T0max = 0.0;          // highest initial temperature
    double env_U = -1.0;              // cached enthalpy_envelope, < 0 when stale
    // ---- batch of independent instances (fem_batch_create); n_inst == 0
    // for a plain mesh.  Ranges are in caller order, [n_inst + 1] each.
    int32_t n_inst = 0;
    std::vector<int64_t> inst_node, inst_elem;
    std::vector<int32_t> inst_plan_order;      // plan position -> caller instance
    std::vector<double> inst_stable, inst_dt;  // stable and chosen time steps
    std::vector<double> inst_t, inst_U0, inst_q; // time, initial energy, boundary heat
    std::vector<int64_t> inst_steps;
    void *dBlkDt = nullptr, *dShDt = nullptr;  // per block / per shared node dt (real)
    std::vector<double> dt_uploaded;           // per-instance dt the two arrays hold
    cudaStream_t own_stream = nullptr;         // graph launches when stream is NULL
    cudaGraphExec_t graph = nullptr;
    std::vector<int64_t> graph_key;            // per-plan-position step counts of graph
    // asynchronous state I/O (fem_set_state_async, fem_get_temperature_async):
    // two device staging buffers each way, a copy stream each way, and
    // events that order every buffer's reuse after its last reader
    cudaGraphExec_t step_graph = nullptr;      // kGraphSteps steps of size step_graph_dt
    double step_graph_dt = 0.0;
    int step_graph_fault = 0;
    cudaStream_t cap_stream = nullptr;         // capture stream of step_graph
    bool async_ok = false;
    cudaStream_t up_stream = nullptr, down_stream = nullptr;
    cudaEvent_t ev_in_ready[2] = {}, ev_in_free[2] = {}, ev_out_ready[2] = {}, ev_out_free[2] = {};
    double *dIn[2] = {nullptr, nullptr}, *dOutT[2] = {nullptr, nullptr};
    int in_idx = 0, out_idx = 0;
};

namespace {

bool finite_all(const double *p, int64_t n)
{
    for (int64_t i = 0; i < n; i++)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Streams and events of the asynchronous I/O; their copies finish first.
// The staging buffers are in m->bufs and go with the other buffers.
void release_async(fem_mesh *m)
{
    for (cudaStream_t s : {m->up_stream, m->down_stream})
        if (s) cudaStreamSynchronize(s);
    for (int i = 0; i < 2; i++)
        for (cudaEvent_t *e : {&m->ev_in_ready[i], &m->ev_in_free[i], &m->ev_out_ready[i], &m->ev_out_free[i]}) {
            if (*e) cudaEventDestroy(*e);
            *e = nullptr;
        }
    for (cudaStream_t *s : {&m->up_stream, &m->down_stream}) {
        if (*s) cudaStreamDestroy(*s);
        *s = nullptr;
    }
    m->dIn[0] = m->dIn[1] = m->dOutT[0] = m->dOutT[1] = nullptr;
    m->in_idx = m->out_idx = 0;
    m->async_ok = false;
}

void release_device(fem_mesh *m)
{
    if (m->device >= 0) cudaSetDevice(m->device);
    release_async(m);
    // a caller's allocator may hand the memory out again at once: let every
    // kernel that uses it finish first
    if (m->free_fn && !m->bufs.empty()) cudaDeviceSynchronize();
    for (auto &b : m->bufs) {
        if (m->free_fn) m->free_fn(b.p, m->alloc_ctx);
        else cudaFree(b.p);
    }
    m->bufs.clear();
    m->dev_bytes = 0;
    m->dev_ok = false;
    m->dE = m->dC = m->dLc = m->dRanges = m->dW = m->dFa = m->dFg = m->dP = m->dT = m->dR = nullptr;
    m->dEloc = m->dCLloc = m->dEsh = nullptr;
    m->dPhloc = nullptr;
    m->dPosloc = m->dHome = m->dMpos = nullptr;
    m->dPh = nullptr;
    m->dBlocks = nullptr;
    m->dShPtr = m->dNodeOld = m->dConn = m->dFconn = nullptr;
    m->dNfPtr = m->dNfIdx = nullptr;
    m->dSched = nullptr;
    m->dEpart = m->dQcum = m->dIo = m->dDirT = m->dOut = nullptr;
    m->dErr = nullptr;
    m->dBlkDt = m->dShDt = nullptr;
    m->dIfPos = m->dIfSis = nullptr;
    m->dIfG = nullptr;
    m->dEmat = nullptr;
    m->dRv = m->dLmC = m->dLmL = m->dLmTs = m->dLmTl = m->dPc = nullptr;
    m->dKtT = m->dKtK = nullptr;
    m->dKtN = nullptr;
    m->dt_uploaded.clear();
    if (m->graph) cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
    if (m->step_graph) cudaGraphExecDestroy(m->step_graph);
    m->step_graph = nullptr;
    if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
    m->cap_stream = nullptr;
    m->graph_key.clear();
    if (m->own_stream) cudaStreamDestroy(m->own_stream);
    m->own_stream = nullptr;
}

bool is_block(const fem_mesh *m);
bool is_lm(const fem_mesh *m);

// With constant k and the enthalpy formulation the block kernel runs with
// 256 threads and reads the conductances from L2 instead of staging them
// in shared memory: a 1,792-tet FP32 block then needs ~56 KB, and four
// CTAs share an SM.  Other thread counts, k(T) and the apparent capacity
// stage the conductances.
bool weights_from_l2(const fem_mesh *m)
{
    return is_block(m) && !is_lm(m) && (m->opt.threads == 0 || m->opt.threads == 256);
}

// Dynamic shared memory of a block-kernel CTA for plan bp (largest block;
// wg: without the conductance rows).
size_t block_smem_of(const BlockPlan &bp, size_t real_size, bool wg)
{
    size_t cw = 0, slots = 0;
    for (const BlockInfo &b : bp.blocks) {
        cw = std::max(cw, (size_t)chunk_words(b));
        slots = std::max(slots, block_slots(b));
    }
    const size_t nes = bp.blocks.empty() ? 8 : (size_t)bp.blocks[0].nep;
    const size_t ls = (bp.max_nloc + 31) / 32 * 32;
    // the slot area also receives the (C, Lc) pairs of the ls local nodes
    slots = (std::max(slots, 2 * ls) + 3) & ~size_t(3);
    return block_kernel_smem(nes, cw, slots, ls, real_size) - (wg ? align16(6 * nes * real_size) : 0);
}

// Four CTAs of the L2-conductance kernel share a GB300 SM (233,472 bytes)
// when each needs at most this much dynamic shared memory (1 KB per CTA is
// reserved, 64 bytes are static).
constexpr size_t kFourCtaSmem = 57216;

int default_block_elems(const fem_mesh *m)
{
    int be = m->opt.block_elems;
    if (be <= 0) be = m->prec == FEM_FP32 ? (weights_from_l2(m) ? 1792 : 2048) : 1024;
    return std::min(std::max(be, 64), 12288);
}

bool is_block(const fem_mesh *m) { return m->opt.variant == FEM_VARIANT_BLOCK; }
bool is_lm(const fem_mesh *m) { return m->opt.formulation == FEM_APPARENT_CAPACITY; }
bool has_dirichlet(const fem_mesh *m) { return !m->is_dir.empty(); }
// Shared-node copies and their mirror positions (block variant; null for
// the flat variants): the set-state kernels write the mirrors themselves.
const int32_t *mirror_ptr(const fem_mesh *m) { return is_block(m) ? m->dShPtr : nullptr; }
const int32_t *mirror_pos(const fem_mesh *m) { return is_block(m) ? m->dMpos : nullptr; }
int64_t mirror_len(const fem_mesh *m) { return is_block(m) ? (int64_t)m->bp.blocks.size() * m->ls : 0; }

// Largest total enthalpy content a stable run of the current data can
// reach: sum_i C_i T_hi + Lc_i, with T_hi the highest temperature the data
// allow (the initial temperatures and the effective ambient T_inf - q/h of
// every Robin face; interface faces take their sisters' temperatures).
// +inf when a face with h = 0 heats by a flux alone (no such bound).
double enthalpy_envelope(fem_mesh *m)
{
    if (m->env_U >= 0.0) return m->env_U;
    double Th = m->acct_T0max;
    for (size_t f = 0; f < m->fa.size(); f++) {
        // fa = h A / 12, fg = A/3 (h T_inf - q): T_inf - q/h = fg / (4 fa)
        if (m->fa[f] > 0.0) Th = std::max(Th, m->fg[f] / (4.0 * m->fa[f]));
        else if (m->fg[f] > 0.0) return m->env_U = HUGE_VAL;
    }
    double U = 0.0;
    for (int64_t i = 0; i < m->N; i++) U += m->Cn[(size_t)i] * Th + m->Lcn[(size_t)i];
    return m->env_U = U;
}

// faces/fa/fg = Robin faces, then interface faces (whose load term the
// interface kernel rewrites every step)
void combine_faces(fem_mesh *m)
{
    m->env_U = -1.0;
    m->faces = m->rb_faces;
    m->faces.insert(m->faces.end(), m->if_faces.begin(), m->if_faces.end());
    m->fa = m->rb_fa;
    m->fa.insert(m->fa.end(), m->if_fa.begin(), m->if_fa.end());
    m->fg = m->rb_fg;
    m->fg.insert(m->fg.end(), (size_t)m->F_if, 0.0);
    m->F = m->F_rb + m->F_if;
}

// Element weights to upload: the constant-k conductances, or with k(T)
// tables those of k = 1 (the kernels scale them by k(mean T)); scale_kmax
// multiplies the latter by each material's largest k (stable-step bound).
std::vector<double> element_weights(const fem_mesh *m, bool scale_kmax)
{
    if (!m->has_kt) return m->w;
    std::vector<double> w((size_t)m->E * 6);
    for (int64_t e = 0; e < m->E; e++) {
        const int32_t *t = &m->tets[4 * (size_t)e];
        double V;
        tet_conductances(&m->xyz[3 * (size_t)t[0]], &m->xyz[3 * (size_t)t[1]], &m->xyz[3 * (size_t)t[2]],
                         &m->xyz[3 * (size_t)t[3]], 1.0, &w[6 * e], &V);
        if (scale_kmax) {
            const int32_t mt = m->mat[e];
            double kmax = m->mat_k[(size_t)mt];
            if (!m->kt_k[(size_t)mt].empty())
                kmax = *std::max_element(m->kt_k[(size_t)mt].begin(), m->kt_k[(size_t)mt].end());
            for (int k = 0; k < 6; k++) w[6 * e + k] *= kmax;
        }
    }
    return w;
}

// caller node ids of the sister face of every interface face [F_if][3]
std::vector<int32_t> sister_nodes(const fem_mesh *m)
{
    std::vector<int32_t> out((size_t)(3 * m->F_if));
    for (int64_t f = 0; f < m->F_if; f++)
        for (int c = 0; c < 3; c++) out[3 * f + c] = m->if_faces[3 * (size_t)m->if_sister[f] + c];
    return out;
}

// number of per-CTA cumulative boundary-heat entries
int64_t n_qcum(const fem_mesh *m)
{
    return is_block(m) ? (int64_t)m->bp.blocks.size() : (int64_t)m->n_node_ctas;
}

// Build the plan (host) if needed.
fem_status ensure_plan(fem_mesh *m)
{
    if (m->plan_ok) return FEM_OK;
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    std::vector<int32_t> owner;
    if (m->F > 0) {
        std::string err = face_owners(m->F, m->faces.data(), m->tets.data(), m->adj, owner);
        if (!err.empty()) return fail(FEM_EINVAL, "%s", err.c_str());
    }
    std::string err;
    try {
        if (is_block(m)) {
            // automatic size with L2 conductances: the largest block has to
            // leave room for four CTAs per SM, else the size shrinks
            const size_t rs = m->prec == FEM_FP32 ? 4 : 8;
            const bool fit = m->opt.block_elems <= 0 && weights_from_l2(m);
            for (int be = default_block_elems(m);; be -= 64) {
                m->bp = BlockPlan();
                err = build_block_plan(m->N, m->E, m->xyz.data(), m->tets.data(), m->rank, m->F,
                                       m->faces.data(), owner, be, (int)rs, m->bp, m->inst_elem,
                                       m->inst_plan_order);
                if (!err.empty() || !fit || be <= 1024 || block_smem_of(m->bp, rs, true) <= kFourCtaSmem)
                    break;
            }
            if (err.empty()) {
                m->blocks_flat.resize(m->bp.blocks.size() * 16);
                std::memcpy(m->blocks_flat.data(), m->bp.blocks.data(),
                            m->bp.blocks.size() * sizeof(BlockInfo));
            }
        } else {
            err = build_flat_plan(m->N, m->E, m->tets.data(), m->rank, m->F,
                                  m->opt.variant == FEM_VARIANT_COLORED, m->fp);
            if (err.empty()) {
                // node -> faces, internal node ids, face positions = caller ids
                m->nf_ptr.assign((size_t)m->N + 1, 0);
                for (int64_t i = 0; i < 3 * m->F; i++) m->nf_ptr[(size_t)m->fp.node_new[m->faces[i]] + 1]++;
                for (int64_t n = 0; n < m->N; n++) m->nf_ptr[n + 1] += m->nf_ptr[n];
                m->nf_idx.assign((size_t)(3 * m->F), 0);
                std::vector<int32_t> fill(m->nf_ptr.begin(), m->nf_ptr.end() - 1);
                for (int64_t f = 0; f < m->F; f++)
                    for (int c = 0; c < 3; c++)
                        m->nf_idx[fill[m->fp.node_new[m->faces[3 * f + c]]]++] = (int32_t)f;
            }
        }
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed while building the plan");
    }
    if (!err.empty()) return fail(FEM_EINVAL, "%s", err.c_str());
    m->plan_ok = true;
    return FEM_OK;
}

const std::vector<int32_t> &node_old_of(const fem_mesh *m)
{
    return is_block(m) ? m->bp.node_old : m->fp.node_old;
}
const std::vector<int32_t> &node_new_of(const fem_mesh *m)
{
    return is_block(m) ? m->bp.node_new : m->fp.node_new;
}

#define CU(call)                                                                            \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            fem_status s_ = e_ == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA;       \
            return fail(s_, "%s failed: %s", #call, cudaGetErrorString(e_));                \
        }                                                                                   \
    } while (0)

#define KERNEL(expr, what)                                                                  \
    do {                                                                                    \
        int e_ = (expr);                                                                    \
        if (e_) return fail(FEM_ECUDA, "%s failed: %s", what, cudaGetErrorString((cudaError_t)e_)); \
    } while (0)

template <typename T>
fem_status upload(fem_mesh *m, T **dst, const T *src, size_t count)
{
    void *p = nullptr;
    const size_t bytes = std::max<size_t>(count, 1) * sizeof(T) + kAllocTailPad;
    cudaError_t e = cudaErrorMemoryAllocation;
    if (alloc_allowed()) {
        if (m->alloc_fn) {   // the caller's allocator (fem_set_allocator)
            p = m->alloc_fn(bytes, m->alloc_ctx);
            e = p ? cudaSuccess : cudaErrorMemoryAllocation;
            if (p && (uintptr_t)p % 256 != 0) {
                m->free_fn(p, m->alloc_ctx);
                return fail(FEM_EINVAL, "the caller's allocator returned a pointer not aligned to 256 bytes");
            }
        } else {
            e = cudaMalloc(&p, bytes);
        }
    }
    if (e != cudaSuccess)
        return fail(e == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA,
                    "device allocation of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
    m->bufs.push_back({p, bytes});
    m->dev_bytes += bytes;
    if (src && count) CU(cudaMemcpy(p, src, count * sizeof(T), cudaMemcpyHostToDevice));
    else CU(cudaMemset(p, 0, bytes));
    *dst = (T *)p;
    return FEM_OK;
}

// Per-node arrays in internal order.
template <typename real>
fem_status upload_nodes(fem_mesh *m)
{
    const auto &old = node_old_of(m);
    std::vector<real> C((size_t)m->N), Lc((size_t)m->N);
    std::vector<uint8_t> ph((size_t)m->N);
    for (int64_t i = 0; i < m->N; i++) {
        int32_t o = old[i];
        C[i] = (real)m->Cn[o];
        Lc[i] = (real)m->Lcn[o];
        ph[i] = (uint8_t)(m->rng_id[o] | (m->is_dir.empty() || !m->is_dir[o] ? 0 : kDirichletBit));
    }
    fem_status st;
    real *p = nullptr;
    if (!is_block(m)) {   // the block variant keeps E in per-block local arrays
        if ((st = upload<real>(m, &p, nullptr, (size_t)m->N))) return st;
        m->dE = p;
    }
    if ((st = upload<real>(m, &p, C.data(), C.size()))) return st;
    m->dC = p;
    if ((st = upload<real>(m, &p, Lc.data(), Lc.size()))) return st;
    m->dLc = p;
    if ((st = upload<uint8_t>(m, &m->dPh, ph.data(), ph.size()))) return st;
    std::vector<real> rg(m->ranges.begin(), m->ranges.end());
    if ((st = upload<real>(m, &p, rg.data(), rg.size()))) return st;
    m->dRanges = p;
    if ((st = upload<int32_t>(m, &m->dNodeOld, old.data(), old.size()))) return st;
    if ((st = upload<double>(m, &m->dIo, nullptr, (size_t)m->N))) return st;
    if ((st = upload<double>(m, &m->dOut, nullptr, 4))) return st;
    if ((st = upload<int>(m, &m->dErr, nullptr, 1))) return st;
    if (!m->is_dir.empty()) {
        std::vector<double> dT((size_t)m->N, 0.0);
        for (int64_t i = 0; i < m->N; i++)
            if (m->is_dir[old[i]]) dT[i] = m->dir_T[old[i]];
        if ((st = upload<double>(m, &m->dDirT, dT.data(), dT.size()))) return st;
    }
    return FEM_OK;
}

// k(T) device tables (every material: its table, or one point at its
// constant k) and the material of every element position (-1: padding ->
// material 0, whose weights are zero there anyway).
template <typename real>
fem_status upload_kt(fem_mesh *m, const std::vector<int32_t> &elem_order)
{
    if (!m->has_kt) {
        if (!is_lm(m)) return FEM_OK;
        std::vector<uint8_t> em(elem_order.size() + 8, 0);
        for (size_t q = 0; q < elem_order.size(); q++)
            if (elem_order[q] >= 0) em[q] = (uint8_t)m->mat[(size_t)elem_order[q]];
        return upload<uint8_t>(m, &m->dEmat, em.data(), em.size());
    }
    std::vector<real> T((size_t)m->n_mat * kKtMax, real(0)), k((size_t)m->n_mat * kKtMax, real(0));
    std::vector<int32_t> n((size_t)m->n_mat);
    for (int32_t mt = 0; mt < m->n_mat; mt++) {
        if (m->kt_T[(size_t)mt].empty()) {
            n[(size_t)mt] = 1;
            k[(size_t)mt * kKtMax] = (real)m->mat_k[(size_t)mt];
        } else {
            n[(size_t)mt] = (int32_t)m->kt_T[(size_t)mt].size();
            for (int32_t j = 0; j < n[(size_t)mt]; j++) {
                T[(size_t)mt * kKtMax + j] = (real)m->kt_T[(size_t)mt][(size_t)j];
                k[(size_t)mt * kKtMax + j] = (real)m->kt_k[(size_t)mt][(size_t)j];
            }
        }
    }
    std::vector<uint8_t> em(elem_order.size() + 8, 0);
    for (size_t q = 0; q < elem_order.size(); q++)
        if (elem_order[q] >= 0) em[q] = (uint8_t)m->mat[(size_t)elem_order[q]];
    fem_status st;
    real *p = nullptr;
    if ((st = upload<real>(m, &p, T.data(), T.size()))) return st;
    m->dKtT = p;
    if ((st = upload<real>(m, &p, k.data(), k.size()))) return st;
    m->dKtK = p;
    if ((st = upload<int32_t>(m, &m->dKtN, n.data(), n.size()))) return st;
    if ((st = upload<uint8_t>(m, &m->dEmat, em.data(), em.size()))) return st;
    return FEM_OK;
}

// Interface faces (Eq. 8): the device position of each one in the face
// arrays (face_order: position -> caller face), its h_i A / 3 and the
// internal ids of its sister's nodes.
template <typename real>
fem_status upload_interface(fem_mesh *m, const std::vector<int32_t> &face_order)
{
    if (m->F_if == 0) return FEM_OK;
    std::vector<int32_t> pos((size_t)m->F_if, -1), sis((size_t)(3 * m->F_if));
    for (size_t q = 0; q < face_order.size(); q++)
        if (face_order[q] >= m->F_rb) pos[(size_t)(face_order[q] - m->F_rb)] = (int32_t)q;
    const auto &nn = node_new_of(m);
    const std::vector<int32_t> sn = sister_nodes(m);
    for (size_t k = 0; k < sn.size(); k++) sis[k] = nn[(size_t)sn[k]];
    for (int32_t v : pos)
        if (v < 0) return fail(FEM_EINVAL, "interface face bookkeeping failed");
    std::vector<real> g(m->if_g.begin(), m->if_g.end());
    fem_status st;
    if ((st = upload<int32_t>(m, &m->dIfPos, pos.data(), pos.size()))) return st;
    if ((st = upload<int32_t>(m, &m->dIfSis, sis.data(), sis.size()))) return st;
    real *p = nullptr;
    if ((st = upload<real>(m, &p, g.data(), g.size()))) return st;
    m->dIfG = p;
    return FEM_OK;
}

template <typename real>
fem_status upload_block(fem_mesh *m)
{
    const BlockPlan &bp = m->bp;
    fem_status st;
    if ((st = upload_nodes<real>(m))) return st;
    // element conductances: block b's six rows at w[(6*b + k)*nes + i]
    // (zero in the padding)
    real *p = nullptr;
    const int32_t nes = bp.blocks.empty() ? 8 : bp.blocks[0].nep;
    m->nes = nes;
    {
        const std::vector<double> src = element_weights(m, false);
        std::vector<real> w((size_t)bp.blocks.size() * 6 * nes, real(0));
        for (size_t bi = 0; bi < bp.blocks.size(); bi++) {
            const BlockInfo &b = bp.blocks[bi];
            for (int32_t i = 0; i < b.ne; i++) {
                int32_t e = bp.elem_order[(size_t)b.e0 + i];
                for (int k = 0; k < 6; k++)
                    w[(6 * bi + k) * (size_t)nes + i] = (real)src[6 * (size_t)e + k];
            }
        }
        if ((st = upload<real>(m, &p, w.data(), w.size()))) return st;
        m->dW = p;
        // apparent capacity: rho V / 4 of element i of block b at b*nes + i,
        // the material table and the capacity partials of shared copies
        if (is_lm(m)) {
            std::vector<real> rv((size_t)bp.blocks.size() * nes + 8, real(0));
            for (size_t bi = 0; bi < bp.blocks.size(); bi++)
                for (int32_t i = 0; i < bp.blocks[bi].ne; i++) {
                    const int32_t e = bp.elem_order[(size_t)bp.blocks[bi].e0 + i];
                    rv[bi * nes + i] = (real)(m->mats[(size_t)m->mat[(size_t)e]].rho * m->vol[(size_t)e] / 4.0);
                }
            if ((st = upload<real>(m, &p, rv.data(), rv.size()))) return st;
            m->dRv = p;
            std::vector<real> c((size_t)m->n_mat), L((size_t)m->n_mat), Ts((size_t)m->n_mat),
                Tl((size_t)m->n_mat);
            for (int32_t mt = 0; mt < m->n_mat; mt++) {
                c[(size_t)mt] = (real)m->mats[(size_t)mt].c;
                L[(size_t)mt] = (real)m->mats[(size_t)mt].latent;
                Ts[(size_t)mt] = (real)m->mats[(size_t)mt].T_solidus;
                Tl[(size_t)mt] = (real)m->mats[(size_t)mt].T_liquidus;
            }
            if ((st = upload<real>(m, &p, c.data(), c.size()))) return st;
            m->dLmC = p;
            if ((st = upload<real>(m, &p, L.data(), L.size()))) return st;
            m->dLmL = p;
            if ((st = upload<real>(m, &p, Ts.data(), Ts.size()))) return st;
            m->dLmTs = p;
            if ((st = upload<real>(m, &p, Tl.data(), Tl.size()))) return st;
            m->dLmTl = p;
            if ((st = upload<real>(m, &p, nullptr, (size_t)std::max<int64_t>(bp.n_copies, 1)))) return st;
            m->dPc = p;
        }
        // k(T) / apparent capacity: the material of element i of block b at b*nes + i
        if (m->has_kt || is_lm(m)) {
            std::vector<int32_t> eo((size_t)bp.blocks.size() * nes, -1);
            for (size_t bi = 0; bi < bp.blocks.size(); bi++)
                for (int32_t i = 0; i < bp.blocks[bi].ne; i++)
                    eo[bi * nes + i] = bp.elem_order[(size_t)bp.blocks[bi].e0 + i];
            if ((st = upload_kt<real>(m, eo))) return st;
        }
    }
    std::vector<real> fa((size_t)bp.F_pad, real(0)), fg((size_t)bp.F_pad, real(0));
    for (int64_t q = 0; q < bp.F_pad; q++) {
        int32_t f = bp.face_order[q];
        if (f < 0) continue;
        fa[q] = (real)m->fa[f];
        fg[q] = (real)m->fg[f];
    }
    if ((st = upload<real>(m, &p, fa.data(), fa.size()))) return st;
    m->dFa = p;
    if ((st = upload<real>(m, &p, fg.data(), fg.size()))) return st;
    m->dFg = p;
    if ((st = upload<BlockInfo>(m, &m->dBlocks, bp.blocks.data(), bp.blocks.size()))) return st;
    {
        // device schedule stream: per block a header of group offsets (in
        // pairs of rounds) and the block's rounds as 32-bit pairs
        std::vector<uint32_t> stream((size_t)bp.n_sched_words, 0u);
        for (const BlockInfo &b : bp.blocks) {
            uint32_t *c = stream.data() + b.s0;
            for (int32_t g = 0; g <= b.ngrp; g++) c[g] = (uint32_t)((bp.grp[(size_t)b.g0 + g] - b.r0) / 2);
            std::memcpy(c + chunk_header_words(b.ngrp), bp.sched.data() + (size_t)b.r0 * 32,
                        (size_t)b.nrounds * 64);
        }
        if ((st = upload<uint32_t>(m, &m->dSched, stream.data(), stream.size()))) return st;
    }
    if ((st = upload<real>(m, &p, nullptr, (size_t)bp.n_copies))) return st;
    m->dP = p;
    if ((st = upload<int32_t>(m, &m->dShPtr, bp.sh_ptr.data(), bp.sh_ptr.size()))) return st;
    {
        // per-block local node arrays at stride ls: interior nodes, then the
        // block's shared copies, then padding; (1/C, Lc) per node, padding
        // (1, 0)
        const int32_t ls = (int32_t)(((int64_t)bp.max_nloc + 31) / 32 * 32);
        m->ls = ls;
        const size_t nl = bp.blocks.size() * (size_t)ls;
        const auto &old = bp.node_old;
        std::vector<real> cl(2 * nl);
        std::vector<uint8_t> ph(nl, 0);
        std::vector<int32_t> pos(nl, 0), home((size_t)std::max<int64_t>(bp.n_int, 1), 0);
        std::vector<int32_t> cloc((size_t)std::max<int64_t>(bp.n_copies, 1), 0);
        for (size_t i = 0; i < nl; i++) { cl[2 * i] = real(1); cl[2 * i + 1] = real(0); }
        auto node_ph = [&](int32_t o) {
            return (uint8_t)(m->rng_id[o] | (m->is_dir.empty() || !m->is_dir[o] ? 0 : kDirichletBit));
        };
        for (size_t bi = 0; bi < bp.blocks.size(); bi++) {
            const BlockInfo &b = bp.blocks[bi];
            const size_t base = bi * (size_t)ls;
            for (int32_t l = 0; l < b.nint; l++) {
                const int32_t o = old[(size_t)b.n0 + l];
                cl[2 * (base + l)] = (real)(1.0 / m->Cn[o]);
                cl[2 * (base + l) + 1] = (real)m->Lcn[o];
                ph[base + l] = node_ph(o);
                home[(size_t)b.n0 + l] = (int32_t)(base + l);
            }
            for (int32_t k = 0; k < b.nsh; k++) {
                const size_t c = (size_t)b.c0 + k, at = base + (size_t)b.nint + k;
                const int32_t o = old[bp.copy_node[c]];
                cl[2 * at] = (real)(1.0 / m->Cn[o]);
                cl[2 * at + 1] = (real)m->Lcn[o];
                ph[at] = node_ph(o);
                pos[at] = bp.copy_pos[c];
                cloc[c] = (int32_t)at;
            }
        }
        std::vector<int32_t> mpos((size_t)std::max<int64_t>(bp.n_copies, 1), 0);
        for (int64_t k = 0; k < bp.n_copies; k++) mpos[k] = cloc[bp.sh_copy[k]];
        if ((st = upload<real>(m, &p, nullptr, nl))) return st;
        m->dEloc = p;
        if ((st = upload<real>(m, &p, cl.data(), cl.size()))) return st;
        m->dCLloc = p;
        if ((st = upload<uint8_t>(m, &m->dPhloc, ph.data(), ph.size()))) return st;
        if ((st = upload<int32_t>(m, &m->dPosloc, pos.data(), pos.size()))) return st;
        if ((st = upload<int32_t>(m, &m->dHome, home.data(), home.size()))) return st;
        if ((st = upload<int32_t>(m, &m->dMpos, mpos.data(), mpos.size()))) return st;
        if ((st = upload<real>(m, &p, nullptr, (size_t)std::max<int64_t>(bp.n_sh, 1)))) return st;
        m->dEsh = p;
    }
    if ((st = upload<double>(m, &m->dEpart, nullptr, 2 * bp.blocks.size()))) return st;
    if ((st = upload<double>(m, &m->dQcum, nullptr, bp.blocks.size()))) return st;
    if (m->n_inst > 0) {   // per-instance time steps of fem_advance
        real *p2 = nullptr;
        if ((st = upload<real>(m, &p2, nullptr, bp.blocks.size()))) return st;
        m->dBlkDt = p2;
        if ((st = upload<real>(m, &p2, nullptr, (size_t)std::max<int64_t>(bp.n_sh, 1)))) return st;
        m->dShDt = p2;
    }
    // kernel configuration: shared memory for the largest block; by default
    // the fewest threads whose 16-byte element accesses cover every block
    size_t cw = 0, slots = 0;
    int32_t max_nep = 0;
    for (const BlockInfo &b : bp.blocks) {
        cw = std::max(cw, (size_t)chunk_words(b));
        slots = std::max(slots, block_slots(b));
        max_nep = std::max(max_nep, b.nep);
    }
    m->chunk_words = (int32_t)cw;
    // the slot area also receives the (C, Lc) pairs of the ls local nodes
    // before pass 1
    slots = std::max(slots, 2 * (size_t)m->ls);
    slots = (slots + 3) & ~size_t(3);
    m->max_slots = (int32_t)slots;
    const int vn = sizeof(real) == 4 ? 4 : 2;
    m->wg = weights_from_l2(m);
    m->threads = m->opt.threads;
    if (m->threads == 0 && m->wg) {
        m->threads = 256;
    } else if (m->threads == 0) {
        m->threads = 128;
        while (m->threads < 1024 && m->threads * vn < max_nep) m->threads *= 2;
    }
    m->smem_bytes = block_smem_of(bp, sizeof(real), m->wg);
    if (m->ls > kMaxLocalNodes)
        return fail(FEM_EINVAL, "a block has %zu local nodes (> %d); lower block_elems", bp.max_nloc,
                    kMaxLocalNodes);
    int dev = 0, optin = 0;
    CU(cudaGetDevice(&dev));
    CU(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    if ((size_t)optin < m->smem_bytes + 1024)
        return fail(FEM_EINVAL, "a block needs %zu bytes of shared memory (device limit %d); lower block_elems",
                    m->smem_bytes, optin);
    KERNEL(configure_block_kernel<real>(m->threads, m->smem_bytes, m->has_kt, is_lm(m), m->wg),
           "configuring the block kernel");
    int per_sm = 0;
    KERNEL(block_kernel_occupancy<real>(m->threads, m->smem_bytes, &per_sm, m->has_kt, is_lm(m), m->wg),
           "occupancy query");
    if (per_sm < 1) return fail(FEM_EINVAL, "the block kernel does not fit on an SM; lower block_elems");
    m->ctas_per_sm = per_sm;
    return upload_interface<real>(m, bp.face_order);
}

template <typename real>
fem_status upload_flat(fem_mesh *m)
{
    const FlatPlan &fp = m->fp;
    fem_status st;
    if ((st = upload_nodes<real>(m))) return st;
    real *p = nullptr;
    {
        const std::vector<double> wsrc = element_weights(m, false);
        std::vector<real> w((size_t)fp.E_pad * 6, real(0));
        std::vector<int32_t> conn((size_t)fp.E_pad * 4, -1);
        for (int64_t q = 0; q < fp.E_pad; q++) {
            int32_t e = fp.elem_order[q];
            if (e < 0) continue;
            for (int k = 0; k < 6; k++) w[(size_t)k * fp.E_pad + q] = (real)wsrc[6 * (size_t)e + k];
            for (int c = 0; c < 4; c++)
                conn[(size_t)c * fp.E_pad + q] = fp.node_new[m->tets[4 * (size_t)e + c]];
        }
        if ((st = upload<real>(m, &p, w.data(), w.size()))) return st;
        m->dW = p;
        if ((st = upload<int32_t>(m, &m->dConn, conn.data(), conn.size()))) return st;
    }
    std::vector<real> fa((size_t)fp.F_pad, real(0)), fg((size_t)fp.F_pad, real(0));
    std::vector<int32_t> fconn((size_t)fp.F_pad * 3, 0);
    for (int64_t q = 0; q < fp.F_pad; q++) {
        int32_t f = fp.face_order[q];
        if (f < 0) continue;
        fa[q] = (real)m->fa[f];
        fg[q] = (real)m->fg[f];
        for (int c = 0; c < 3; c++)
            fconn[(size_t)c * fp.F_pad + q] = fp.node_new[m->faces[3 * (size_t)f + c]];
    }
    if ((st = upload<real>(m, &p, fa.data(), fa.size()))) return st;
    m->dFa = p;
    if ((st = upload<real>(m, &p, fg.data(), fg.size()))) return st;
    m->dFg = p;
    if ((st = upload<int32_t>(m, &m->dFconn, fconn.data(), fconn.size()))) return st;
    if ((st = upload<int32_t>(m, &m->dNfPtr, m->nf_ptr.data(), m->nf_ptr.size()))) return st;
    if ((st = upload<int32_t>(m, &m->dNfIdx, m->nf_idx.data(), m->nf_idx.size()))) return st;
    if ((st = upload<real>(m, &p, nullptr, (size_t)m->N))) return st;
    m->dT = p;
    if ((st = upload<real>(m, &p, nullptr, (size_t)m->N))) return st;
    m->dR = p;
    m->n_node_ctas = (int)std::max<int64_t>(1, (m->N + 255) / 256);
    if ((st = upload<double>(m, &m->dEpart, nullptr, 2 * (size_t)m->n_node_ctas))) return st;
    if ((st = upload<double>(m, &m->dQcum, nullptr, (size_t)m->n_node_ctas))) return st;
    if ((st = upload_kt<real>(m, fp.elem_order))) return st;
    return upload_interface<real>(m, fp.face_order);
}

template <typename real>
BlockArgs<real> block_args(const fem_mesh *m)
{
    BlockArgs<real> a{};
    a.blocks = m->dBlocks;
    a.n_blocks = (int32_t)m->bp.blocks.size();
    a.ls = m->ls;
    a.Eloc = (real *)m->dEloc;
    a.CLloc = (const real *)m->dCLloc;
    a.phloc = m->dPhloc;
    a.posloc = m->dPosloc;
    a.ranges = (const real *)m->dRanges;
    a.w = (const real *)m->dW;
    a.nes = m->nes;
    a.fa = (const real *)m->dFa;
    a.fg = (const real *)m->dFg;
    a.sched = m->dSched;
    a.chunk_words = m->chunk_words;
    a.max_slots = m->max_slots;
    a.P = (real *)m->dP;
    a.sh_ptr = m->dShPtr;
    a.mpos = m->dMpos;
    a.Esh = (real *)m->dEsh;
    a.ph = m->dPh;
    a.n_int = m->bp.n_int;
    a.n_sh = m->bp.n_sh;
    a.n_copies = m->bp.n_copies;
    a.qcum = m->dQcum;
    a.err = m->dErr;
    a.b_first = 0;
    a.b_count = (int32_t)m->bp.blocks.size();
    a.s_first = 0;
    a.s_end = m->bp.n_sh;
    a.blk_dt = nullptr;
    a.sh_dt = nullptr;
    a.emat = m->dEmat;
    a.kt_T = (const real *)m->dKtT;
    a.kt_k = (const real *)m->dKtK;
    a.kt_n = m->dKtN;
    a.rv = (const real *)m->dRv;
    a.lm_c = (const real *)m->dLmC;
    a.lm_L = (const real *)m->dLmL;
    a.lm_Ts = (const real *)m->dLmTs;
    a.lm_Tl = (const real *)m->dLmTl;
    a.Pc = (real *)m->dPc;
    // test hook: a bounded wait that runs out (see BlockArgs)
    const char *skip = getenv("FEM_FAULT_SKIP_WEIGHT_COPY");
    a.fault_skip_weights = (skip && *skip && *skip != '0') ? 1 : 0;
    return a;
}

// Where E of internal node i lives (see StateView).
template <typename real>
StateView<real> view_of(const fem_mesh *m)
{
    StateView<real> v{};
    if (is_block(m)) {
        v.Eloc = (real *)m->dEloc;
        v.Esh = (real *)m->dEsh;
        v.home = m->dHome;
        v.n_int = m->bp.n_int;
    } else {
        v.Eloc = (real *)m->dE;
        v.n_int = m->N;
    }
    v.is_T = m->opt.formulation == FEM_APPARENT_CAPACITY;
    v.C = (const real *)m->dC;
    v.Lc = (const real *)m->dLc;
    v.ph = m->dPh;
    v.ranges = (const real *)m->dRanges;
    return v;
}

template <typename real>
FlatArgs<real> flat_args(const fem_mesh *m)
{
    FlatArgs<real> a{};
    a.E = (real *)m->dE;
    a.C = (const real *)m->dC;
    a.Lc = (const real *)m->dLc;
    a.ph = m->dPh;
    a.ranges = (const real *)m->dRanges;
    a.n_nodes = m->N;
    a.T = (real *)m->dT;
    a.R = (real *)m->dR;
    a.conn = m->dConn;
    a.w = (const real *)m->dW;
    a.n_elems = m->E;
    a.e_stride = m->fp.E_pad;
    a.fconn = m->dFconn;
    a.fa = (const real *)m->dFa;
    a.fg = (const real *)m->dFg;
    a.n_faces = m->F;
    a.f_stride = m->fp.F_pad;
    a.qcum = m->dQcum;
    a.emat = m->dEmat;
    a.kt_T = (const real *)m->dKtT;
    a.kt_k = (const real *)m->dKtK;
    a.kt_n = m->dKtN;
    a.err = m->dErr;
    return a;
}

// Number of CTAs (and FP64 partial pairs) of the whole-state energy
// snapshot; bounded by the size of the per-step partial array it reuses.
int snapshot_ctas(const fem_mesh *m)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(n_qcum(m), 152 * 4));
}

// FP64 sums of the current state into m->dOut: {sum E, latent, sum qcum}.
template <typename real>
int energy_snapshot(fem_mesh *m)
{
    const int nct = snapshot_ctas(m);
    int e = launch_energy_snapshot<real>(view_of<real>(m), (const real *)m->dC,
                                         (const real *)m->dLc, m->dPh, (const real *)m->dRanges,
                                         m->N, m->dEpart, nct, m->stream);
    if (!e) e = launch_energy_reduce(m->dEpart, nct, nullptr, 0, m->dQcum, n_qcum(m), m->dOut, m->stream);
    return e;
}

// Block variant: the block-ordered copies of shared nodes' E follow a state
// that was set from outside.
template <typename real>
int refresh_mirror(fem_mesh *m)
{
    if (!is_block(m)) return 0;
    return launch_mirror_copies<real>(block_args<real>(m), m->stream);
}

// Sum of E over every instance's nodes (FP64, ascending caller node order),
// from the device state.  Synchronises.
template <typename real>
fem_status instance_sums(fem_mesh *m, std::vector<double> &U)
{
    std::vector<double> E((size_t)m->N);
    KERNEL(launch_get_state<real>(view_of<real>(m), m->dIo, m->dNodeOld, m->N, m->stream),
           "read-back kernel");
    CU(cudaMemcpyAsync(E.data(), m->dIo, (size_t)m->N * sizeof(double), cudaMemcpyDeviceToHost,
                       m->stream));
    CU(cudaStreamSynchronize(m->stream));
    U.assign((size_t)m->n_inst, 0.0);
    for (int32_t i = 0; i < m->n_inst; i++)
        for (int64_t n = m->inst_node[(size_t)i]; n < m->inst_node[(size_t)i + 1]; n++)
            U[(size_t)i] += E[(size_t)n];
    return FEM_OK;
}

// Upload of a caller-order E array already on the device (src, io = double
// or float); the block variant's kernel also writes the shared nodes'
// mirrors.
template <typename real, typename io>
int launch_upload(fem_mesh *m, const io *src)
{
    if constexpr (sizeof(io) == 8)
        return launch_set_state<real>(view_of<real>(m), (const double *)src, m->dNodeOld, m->N, m->dErr,
                                      m->stream, mirror_ptr(m), mirror_pos(m), mirror_len(m));
    else
        return launch_set_state_f32<real>(view_of<real>(m), (const float *)src, m->dNodeOld, m->N, m->dErr,
                                          m->stream, mirror_ptr(m), mirror_pos(m), mirror_len(m));
}

// Apply a pending initial condition or checkpoint on the device.
template <typename real>
fem_status apply_pending(fem_mesh *m)
{
    if (m->state != fem_mesh::ST_PENDING_T && m->state != fem_mesh::ST_PENDING_E) return FEM_OK;
    CU(cudaMemcpyAsync(m->dIo, m->pending.data(), (size_t)m->N * sizeof(double),
                       cudaMemcpyHostToDevice, m->stream));
    const bool initial = m->state == fem_mesh::ST_PENDING_T;
    if (initial)
        KERNEL(launch_set_temperature<real>(view_of<real>(m), (const real *)m->dC, (const real *)m->dLc,
                                            m->dPh, (const real *)m->dRanges, m->dIo, m->dNodeOld,
                                            m->dDirT, m->N, m->stream),
               "initial-state kernel");
    else
        KERNEL((launch_upload<real, double>(m, m->dIo)),
               "state kernel");
    if (initial) KERNEL(refresh_mirror<real>(m), "mirror kernel");
    CU(cudaMemsetAsync(m->dQcum, 0, (size_t)n_qcum(m) * sizeof(double), m->stream));
    if (initial) {
        // a new energy account: U0 = sum E of the initial state, no boundary heat
        KERNEL(energy_snapshot<real>(m), "energy kernel");
        double out[3];
        CU(cudaMemcpyAsync(out, m->dOut, 3 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
        CU(cudaStreamSynchronize(m->stream));
        m->U0 = out[0];
        m->q_carry = 0.0;
        if (m->n_inst > 0) {   // per-instance energy accounts
            fem_status st = instance_sums<real>(m, m->inst_U0);
            if (st) return st;
            m->inst_q.assign((size_t)m->n_inst, 0.0);
        }
    } else {
        CU(cudaStreamSynchronize(m->stream));
    }
    m->state = fem_mesh::ST_DEVICE;
    std::vector<double>().swap(m->pending);
    return FEM_OK;
}

fem_status ensure_device(fem_mesh *m)
{
    fem_status st = ensure_plan(m);
    if (st) return st;
    if (m->dev_ok) return FEM_OK;
    int ndev = 0;
    cudaError_t ce = cudaGetDeviceCount(&ndev);
    if (ce != cudaSuccess || ndev == 0)
        return fail(FEM_ECUDA, "no CUDA device available (%s)", cudaGetErrorString(ce));
    CU(cudaGetDevice(&m->device));
    g_alloc_count = 0;
    if (is_block(m))
        st = m->prec == FEM_FP32 ? upload_block<float>(m) : upload_block<double>(m);
    else
        st = m->prec == FEM_FP32 ? upload_flat<float>(m) : upload_flat<double>(m);
    if (st) {
        std::string keep = g_err;
        release_device(m);
        g_err = keep;
        return st;
    }
    m->dev_ok = true;
    return FEM_OK;
}

// Copy the device state back to a host checkpoint (before a plan rebuild),
// so set_* calls after stepping keep the current state and energy account.
fem_status stash_state(fem_mesh *m)
{
    if (!m->dev_ok || m->state != fem_mesh::ST_DEVICE) return FEM_OK;
    cudaSetDevice(m->device);
    std::vector<double> E((size_t)m->N);
    KERNEL(m->prec == FEM_FP32
               ? launch_get_state<float>(view_of<float>(m), m->dIo, m->dNodeOld, m->N, m->stream)
               : launch_get_state<double>(view_of<double>(m), m->dIo, m->dNodeOld, m->N, m->stream),
           "state read-back");
    CU(cudaMemcpyAsync(E.data(), m->dIo, (size_t)m->N * sizeof(double), cudaMemcpyDeviceToHost,
                       m->stream));
    KERNEL(launch_energy_reduce(m->dEpart, 0, nullptr, 0, m->dQcum, n_qcum(m), m->dOut, m->stream),
           "energy kernel");
    double r[3];
    CU(cudaMemcpyAsync(r, m->dOut, 3 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    m->q_carry += r[2];
    m->pending.swap(E);
    m->state = fem_mesh::ST_PENDING_E;
    return FEM_OK;
}

fem_status invalidate_plan(fem_mesh *m)
{
    fem_status st = stash_state(m);
    if (st) return st;
    release_device(m);
    m->plan_ok = false;
    m->bp = BlockPlan();
    m->fp = FlatPlan();
    return FEM_OK;
}

// Kernels of one step, in launch order: {interface faces, when there are
// any}, then block variant {block step, shared update}; flat variants
// {temperatures, element pass, node update}.
int step_kernel_count(const fem_mesh *m) { return (is_block(m) ? 2 : 3) + (m->F_if > 0 ? 1 : 0); }

template <typename real>
fem_status launch_interface_kernel(fem_mesh *m, cudaStream_t st)
{
    KERNEL(launch_interface<real>(view_of<real>(m), (const real *)m->dC, (const real *)m->dLc, m->dPh,
                                  (const real *)m->dRanges, (real *)m->dFg, m->dIfPos, m->dIfSis,
                                  (const real *)m->dIfG, m->F_if, st),
           "interface kernel");
    return FEM_OK;
}

template <typename real>
fem_status launch_step_kernel(fem_mesh *m, int k, double dt, cudaStream_t st)
{
    if (m->F_if > 0) {
        if (k == 0) return launch_interface_kernel<real>(m, st);
        k--;
    }
    if (is_block(m)) {
        const BlockArgs<real> a = block_args<real>(m);
        if (k == 0)
            KERNEL(launch_block_kernel<real>(a, m->threads, m->smem_bytes, dt, st, m->has_kt,
                                             is_lm(m), m->wg),
                   "block kernel");
        else
            KERNEL(launch_shared_update<real>(a, dt, st), "shared-node kernel");
    } else {
        const FlatArgs<real> a = flat_args<real>(m);
        if (k == 0)
            KERNEL(launch_flat_temperature<real>(a, st), "temperature kernel");
        else if (k == 1)
            KERNEL(launch_flat_elements<real>(a, m->opt.variant == FEM_VARIANT_ATOMIC,
                                              m->fp.color_start.data(), m->fp.n_colors, st),
                   "element kernel");
        else
            KERNEL(launch_flat_update<real>(a, m->dNfPtr, m->dNfIdx, m->n_node_ctas, dt, st),
                   "update kernel");
    }
    return FEM_OK;
}

constexpr int64_t kGraphSteps = 32;   // steps per captured graph

// The launches of kGraphSteps steps of size dt, captured once into a graph
// (on a private stream) and replayed on the mesh's stream: a small mesh's
// step is a few tens of microseconds, of which launch gaps are a visible part.
template <typename real>
fem_status ensure_step_graph(fem_mesh *m, double dt)
{
    const char *skip = std::getenv("FEM_FAULT_SKIP_WEIGHT_COPY");
    const int fault = (skip && *skip && *skip != '0') ? 1 : 0;
    if (m->step_graph && m->step_graph_dt == dt && m->step_graph_fault == fault) return FEM_OK;
    if (m->step_graph) cudaGraphExecDestroy(m->step_graph);
    m->step_graph = nullptr;
    if (!m->cap_stream) CU(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    CU(cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal));
    const int nk = step_kernel_count(m);
    fem_status st = FEM_OK;
    for (int64_t s = 0; s < kGraphSteps && !st; s++)
        for (int k = 0; k < nk && !st; k++) st = launch_step_kernel<real>(m, k, dt, m->cap_stream);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(m->cap_stream, &g);
    if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ce != cudaSuccess) return fail(FEM_ECUDA, "step graph capture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&m->step_graph, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        m->step_graph = nullptr;
        return fail(FEM_ECUDA, "step graph instantiation: %s", cudaGetErrorString(ie));
    }
    m->step_graph_dt = dt;
    m->step_graph_fault = fault;
    return FEM_OK;
}

template <typename real>
fem_status step_impl(fem_mesh *m, int64_t n, double dt)
{
    const int nk = step_kernel_count(m);
    int64_t done = 0;
    if (n >= kGraphSteps) {
        fem_status st = ensure_step_graph<real>(m, dt);
        if (st) return st;
        for (; done + kGraphSteps <= n; done += kGraphSteps)
            CU(cudaGraphLaunch(m->step_graph, m->stream));
    }
    for (int64_t s = done; s < n; s++)
        for (int k = 0; k < nk; k++) {
            fem_status st = launch_step_kernel<real>(m, k, dt, m->stream);
            if (st) return st;
        }
    m->step += n;
    m->acct_steps += n;
    m->time += dt * (double)n;
    return FEM_OK;
}

// As step_impl, with CUDA events around every kernel; ms[k] accumulates
// the device time of kernel k.
template <typename real>
fem_status step_profile_impl(fem_mesh *m, int64_t n, double dt, double *ms)
{
    const int nk = step_kernel_count(m);
    cudaEvent_t ev[4];
    for (int k = 0; k <= nk; k++) CU(cudaEventCreate(&ev[k]));
    fem_status st = FEM_OK;
    for (int64_t s = 0; s < n && st == FEM_OK; s++) {
        for (int k = 0; k < nk && st == FEM_OK; k++) {
            cudaEventRecord(ev[k], m->stream);
            st = launch_step_kernel<real>(m, k, dt, m->stream);
        }
        if (st) break;
        cudaEventRecord(ev[nk], m->stream);
        if (cudaEventSynchronize(ev[nk]) != cudaSuccess) {
            st = fail(FEM_ECUDA, "event synchronisation failed");
            break;
        }
        for (int k = 0; k < nk; k++) {
            float t = 0.f;
            cudaEventElapsedTime(&t, ev[k], ev[k + 1]);
            ms[k] += t;
        }
        m->step += 1;
        m->acct_steps += 1;
        m->time += dt;
    }
    for (int k = 0; k <= nk; k++) cudaEventDestroy(ev[k]);
    return st;
}

// Device error flag (kErr* bits): a bounded wait that gave up, a non-finite
// value given to fem_set_state, a non-finite temperature read back.  The
// stream is synchronised; the flag is cleared once reported.
fem_status check_device_flag(fem_mesh *m)
{
    if (!m->dErr) return FEM_OK;
    int flag = 0;
    CU(cudaMemcpyAsync(&flag, m->dErr, sizeof(int), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    if (!flag) return FEM_OK;
    CU(cudaMemsetAsync(m->dErr, 0, sizeof(int), m->stream));
    if (flag & kErrWaitTimeout)
        return fail(FEM_ETIMEOUT, "a bounded device wait gave up; the state is not valid");
    if (flag & kErrBadIndex)
        return fail(FEM_ECUDA, "a device index failed its bounds check (checked build)");
    if (flag & kErrBadInput)
        return fail(FEM_EINVAL, "fem_set_state received a non-finite enthalpy");
    return fail(FEM_EUNSTABLE, "non-finite temperature: dt above the stable limit?");
}

fem_status ready_for_io(fem_mesh *m)
{
    if (m->state == fem_mesh::ST_NONE) return fail(FEM_ESTATE, "no initial state (call fem_set_temperature)");
    fem_status st = ensure_device(m);
    if (st) return st;
    cudaSetDevice(m->device);
    return m->prec == FEM_FP32 ? apply_pending<float>(m) : apply_pending<double>(m);
}

// Batches: add every block's cumulative boundary heat to its instance's
// account (before the device buffers are released).
fem_status fold_instance_heat(fem_mesh *m)
{
    if (m->n_inst == 0 || !m->dev_ok || m->state != fem_mesh::ST_DEVICE) return FEM_OK;
    std::vector<double> q(m->bp.blocks.size());
    CU(cudaMemcpyAsync(q.data(), m->dQcum, q.size() * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    for (size_t b = 0; b < q.size(); b++) m->inst_q[(size_t)m->bp.block_inst[b]] += q[b];
    return FEM_OK;
}

// Drop the device data and the partition; the next ready_for_io rebuilds
// both from the options and uploads E (caller order) as the state.
void reset_partition(fem_mesh *m, const std::vector<double> &E)
{
    release_device(m);
    m->plan_ok = false;
    m->bp = BlockPlan();
    m->pending = E;
    m->state = fem_mesh::ST_PENDING_E;
}

// Mean device ms per step of `steps` steps after two warm-up steps.
template <typename real>
fem_status time_steps(fem_mesh *m, int32_t steps, double dt, double *ms)
{
    fem_status st = step_impl<real>(m, 2, dt);
    if (st) return st;
    cudaEvent_t e0, e1;
    CU(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(FEM_ECUDA, "event creation failed");
    }
    cudaEventRecord(e0, m->stream);
    st = step_impl<real>(m, steps, dt);
    cudaEventRecord(e1, m->stream);
    float t = 0.f;
    if (!st && (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t, e0, e1) != cudaSuccess))
        st = fail(FEM_ECUDA, "event timing failed");
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st) return st;
    *ms = (double)t / (double)steps;
    return check_device_flag(m);
}

fem_status ensure_async(fem_mesh *m)
{
    if (m->async_ok) return FEM_OK;
    for (int i = 0; i < 2; i++) {
        fem_status st = upload<double>(m, &m->dIn[i], nullptr, (size_t)m->N);
        if (!st) st = upload<double>(m, &m->dOutT[i], nullptr, (size_t)m->N);
        if (st) return st;
    }
    CU(cudaStreamCreateWithFlags(&m->up_stream, cudaStreamNonBlocking));
    CU(cudaStreamCreateWithFlags(&m->down_stream, cudaStreamNonBlocking));
    for (int i = 0; i < 2; i++)
        for (cudaEvent_t *e : {&m->ev_in_ready[i], &m->ev_in_free[i], &m->ev_out_ready[i], &m->ev_out_free[i]})
            CU(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    m->async_ok = true;
    return FEM_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char *fem_last_error(void) { return g_err.c_str(); }

fem_status fem_mesh_create_ex(const double *xyz, int64_t n_nodes, const int32_t *tets,
                              int64_t n_tets, const int32_t *mat_id, fem_precision prec,
                              int reorder, const fem_options *opts, fem_mesh **out)
{
    if (!out) return fail(FEM_EINVAL, "out is NULL");
    *out = nullptr;
    if (n_nodes <= 0 || n_tets <= 0) return fail(FEM_EINVAL, "n_nodes and n_tets must be positive");
    if (n_nodes > INT32_MAX - 1 || n_tets > INT32_MAX / 8)
        return fail(FEM_EINVAL, "mesh too large for 32-bit ids");
    if (!xyz || !tets || !mat_id) return fail(FEM_EINVAL, "NULL array argument");
    if (prec != FEM_FP64 && prec != FEM_FP32) return fail(FEM_EINVAL, "unknown precision %d", (int)prec);
    if (reorder != 0 && reorder != 1) return fail(FEM_EINVAL, "reorder must be 0 or 1");
    fem_options opt{};
    if (opts) opt = *opts;
    if (opt.variant < 0 || opt.variant > 2) return fail(FEM_EINVAL, "unknown variant %d", opt.variant);
    if (opt.formulation != FEM_ENTHALPY && opt.formulation != FEM_APPARENT_CAPACITY)
        return fail(FEM_EINVAL, "unknown formulation %d", opt.formulation);
    if (opt.formulation == FEM_APPARENT_CAPACITY && opt.variant != FEM_VARIANT_BLOCK)
        return fail(FEM_EINVAL, "the apparent-capacity formulation uses the block variant");
    if (opt.threads != 0 && opt.threads != 128 && opt.threads != 256 && opt.threads != 512 &&
        opt.threads != 1024)
        return fail(FEM_EINVAL, "threads must be 0, 128, 256, 512 or 1024");
    std::unique_ptr<fem_mesh> m;
    try {
        if (!finite_all(xyz, 3 * n_nodes)) return fail(FEM_EINVAL, "non-finite coordinate");
        m.reset(new fem_mesh());
        m->N = n_nodes;
        m->E = n_tets;
        m->prec = prec;
        m->reorder = reorder;
        m->opt = opt;
        m->xyz.assign(xyz, xyz + 3 * n_nodes);
        m->tets.assign(tets, tets + 4 * n_tets);
        m->mat.assign(mat_id, mat_id + n_tets);
        m->vol.resize((size_t)n_tets);
        for (int64_t e = 0; e < n_tets; e++) {
            const int32_t *t = tets + 4 * e;
            for (int c = 0; c < 4; c++)
                if (t[c] < 0 || t[c] >= n_nodes)
                    return fail(FEM_EINVAL, "tet %lld corner %d: node id %d out of range",
                                (long long)e, c, t[c]);
            for (int c = 0; c < 4; c++)
                for (int d = c + 1; d < 4; d++)
                    if (t[c] == t[d]) return fail(FEM_EINVAL, "tet %lld repeats node %d", (long long)e, t[c]);
            if (mat_id[e] < 0) return fail(FEM_EINVAL, "tet %lld has negative material id", (long long)e);
            const double *x[4];
            for (int c = 0; c < 4; c++) x[c] = xyz + 3 * (size_t)t[c];
            double V = tet_signed_volume(x[0], x[1], x[2], x[3]);
            double l = 0.0;
            for (int c = 0; c < 4; c++)
                for (int d = c + 1; d < 4; d++) {
                    double dx = x[c][0] - x[d][0], dy = x[c][1] - x[d][1], dz = x[c][2] - x[d][2];
                    l += std::sqrt(dx * dx + dy * dy + dz * dz);
                }
            l /= 6.0;
            if (std::fabs(V) < 1e-12 * l * l * l)
                return fail(FEM_EINVAL, "tet %lld is degenerate (volume %g)", (long long)e, V);
            m->vol[e] = std::fabs(V);
        }
        build_node_elems(n_nodes, n_tets, tets, m->adj);
        for (int64_t n = 0; n < n_nodes; n++)
            if (m->adj.ptr[n + 1] == m->adj.ptr[n])
                return fail(FEM_EINVAL, "node %lld belongs to no tet", (long long)n);
        m->bw_input = mesh_bandwidth(n_tets, tets, nullptr);
        if (reorder) {
            rcm_order(n_nodes, n_tets, tets, m->adj, m->rank);
            m->bw_rank = mesh_bandwidth(n_tets, tets, m->rank.data());
        } else {
            m->rank.resize((size_t)n_nodes);
            for (int64_t n = 0; n < n_nodes; n++) m->rank[n] = (int32_t)n;
            m->bw_rank = m->bw_input;
        }
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    *out = m.release();
    return ok();
}

fem_status fem_mesh_create(const double *xyz, int64_t n_nodes, const int32_t *tets, int64_t n_tets,
                           const int32_t *mat_id, fem_precision prec, int reorder, fem_mesh **out)
{
    return fem_mesh_create_ex(xyz, n_nodes, tets, n_tets, mat_id, prec, reorder, nullptr, out);
}

void fem_mesh_destroy(fem_mesh *m)
{
    if (!m) return;
    release_device(m);
    delete m;
}

fem_status fem_set_materials(fem_mesh *m, const fem_material *mats, int32_t n_mat)
{
    if (!m || !mats) return fail(FEM_EINVAL, "NULL argument");
    if (n_mat <= 0) return fail(FEM_EINVAL, "n_mat must be positive");
    if (m->n_inst > 0) return fail(FEM_ESTATE, "a batch takes its materials and boundaries from its parts");
    for (int32_t i = 0; i < n_mat; i++) {
        const fem_material &q = mats[i];
        double v[6] = {q.rho, q.c, q.k, q.latent, q.T_solidus, q.T_liquidus};
        if (!finite_all(v, 6)) return fail(FEM_EINVAL, "material %d has a non-finite value", i);
        if (q.rho <= 0 || q.c <= 0 || q.k <= 0)
            return fail(FEM_EINVAL, "material %d: rho, c and k must be positive", i);
        if (q.latent < 0) return fail(FEM_EINVAL, "material %d: negative latent heat", i);
        if (q.latent > 0 && q.T_liquidus < q.T_solidus)
            return fail(FEM_EINVAL, "material %d: T_liquidus < T_solidus", i);
        if (q.latent > 0 && is_lm(m) && !(q.T_liquidus > q.T_solidus))
            return fail(FEM_EINVAL, "material %d: the apparent-capacity formulation needs "
                                    "T_liquidus > T_solidus", i);
    }
    for (int64_t e = 0; e < m->E; e++)
        if (m->mat[e] >= n_mat)
            return fail(FEM_EINVAL, "tet %lld has material id %d >= n_mat", (long long)e, m->mat[e]);
    try {
        std::vector<double> w((size_t)m->E * 6), C((size_t)m->N, 0.0), mn((size_t)m->N, 0.0),
            Lc((size_t)m->N, 0.0);
        std::vector<uint8_t> rid((size_t)m->N, 0), has((size_t)m->N, 0);
        // distinct (Ts, Tl) ranges of the phase-change materials
        std::vector<double> ranges;
        std::vector<int> mat_range((size_t)n_mat, -1);
        for (int32_t i = 0; i < n_mat; i++) {
            if (mats[i].latent <= 0) continue;
            int found = -1;
            for (size_t r = 0; r < ranges.size() / 2; r++)
                if (ranges[2 * r] == mats[i].T_solidus && ranges[2 * r + 1] == mats[i].T_liquidus)
                    found = (int)r;
            if (found < 0) {
                if ((int)(ranges.size() / 2) >= kMaxRanges)
                    return fail(FEM_EINVAL, "more than %d distinct phase-change ranges", kMaxRanges);
                found = (int)(ranges.size() / 2);
                ranges.push_back(mats[i].T_solidus);
                ranges.push_back(mats[i].T_liquidus);
            }
            mat_range[i] = found;
        }
        if (ranges.empty()) { ranges.push_back(0.0); ranges.push_back(0.0); }
        for (int64_t e = 0; e < m->E; e++) {
            const fem_material &q = mats[m->mat[e]];
            const int32_t *t = &m->tets[4 * (size_t)e];
            double V;
            tet_conductances(&m->xyz[3 * (size_t)t[0]], &m->xyz[3 * (size_t)t[1]],
                             &m->xyz[3 * (size_t)t[2]], &m->xyz[3 * (size_t)t[3]], q.k, &w[6 * e], &V);
            // row-sum lumping: each corner gets a quarter of rho c V
            for (int c = 0; c < 4; c++) {
                int32_t n = t[c];
                C[n] += q.rho * q.c * V / 4.0;
                mn[n] += q.rho * V / 4.0;
                if (q.latent > 0) {
                    int r = mat_range[m->mat[e]];
                    if (has[n] && rid[n] != r)
                        return fail(FEM_EINVAL,
                                    "node %d touches phase-change materials with different ranges", n);
                    rid[n] = (uint8_t)r;
                    has[n] = 1;
                    Lc[n] += q.rho * q.latent * V / 4.0;
                }
            }
        }
        fem_status st = invalidate_plan(m);
        if (st) return st;
        m->w.swap(w);
        m->Cn.swap(C);
        m->env_U = -1.0;
        m->mn.swap(mn);
        m->Lcn.swap(Lc);
        m->rng_id.swap(rid);
        m->ranges.swap(ranges);
        m->n_mat = n_mat;
        m->mats.assign(mats, mats + n_mat);
        m->mat_k.resize((size_t)n_mat);
        for (int32_t i = 0; i < n_mat; i++) m->mat_k[(size_t)i] = mats[i].k;
        m->kt_T.assign((size_t)n_mat, {});
        m->kt_k.assign((size_t)n_mat, {});
        m->has_kt = false;
        m->have_mat = true;
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    return ok();
}

fem_status fem_set_boundary(fem_mesh *m, const int32_t *faces, int64_t n_faces, const double *h,
                            const double *T_inf, const double *q)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (n_faces < 0) return fail(FEM_EINVAL, "n_faces must be >= 0");
    if (m->n_inst > 0) return fail(FEM_ESTATE, "a batch takes its materials and boundaries from its parts");
    if (n_faces > 0 && (!faces || !h || !T_inf)) return fail(FEM_EINVAL, "NULL array argument");
    if (n_faces > INT32_MAX / 3) return fail(FEM_EINVAL, "too many faces");
    std::vector<int32_t> fc;
    std::vector<double> fa, fg;
    try {
        if (n_faces > 0) fc.assign(faces, faces + 3 * n_faces);
        fa.resize((size_t)n_faces);
        fg.resize((size_t)n_faces);
        for (int64_t f = 0; f < n_faces; f++) {
            for (int c = 0; c < 3; c++)
                if (fc[3 * f + c] < 0 || fc[3 * f + c] >= m->N)
                    return fail(FEM_EINVAL, "face %lld: node id out of range", (long long)f);
            double qq = q ? q[f] : 0.0;
            if (!std::isfinite(h[f]) || !std::isfinite(T_inf[f]) || !std::isfinite(qq))
                return fail(FEM_EINVAL, "face %lld: non-finite h, T_inf or q", (long long)f);
            if (h[f] < 0) return fail(FEM_EINVAL, "face %lld: negative h", (long long)f);
            const double *xa = &m->xyz[3 * (size_t)fc[3 * f]], *xb = &m->xyz[3 * (size_t)fc[3 * f + 1]],
                         *xc = &m->xyz[3 * (size_t)fc[3 * f + 2]];
            double u[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
            double v[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
            double nx = u[1] * v[2] - u[2] * v[1], ny = u[2] * v[0] - u[0] * v[2],
                   nz = u[0] * v[1] - u[1] * v[0];
            double A = 0.5 * std::sqrt(nx * nx + ny * ny + nz * nz);
            fa[f] = h[f] * A / 12.0;
            fg[f] = A / 3.0 * (h[f] * T_inf[f] - qq);
        }
        std::vector<int32_t> owner;
        std::string err = face_owners(n_faces, fc.data(), m->tets.data(), m->adj, owner);
        if (!err.empty()) return fail(FEM_EINVAL, "%s", err.c_str());
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    fem_status st = invalidate_plan(m);
    if (st) return st;
    m->rb_faces.swap(fc);
    m->rb_fa.swap(fa);
    m->rb_fg.swap(fg);
    m->F_rb = n_faces;
    combine_faces(m);
    return ok();
}

fem_status fem_set_conductivity(fem_mesh *m, int32_t mat, int32_t n, const double *T,
                                const double *k)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (m->n_inst > 0) return fail(FEM_ESTATE, "a batch takes its materials and boundaries from its parts");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    if (mat < 0 || mat >= m->n_mat) return fail(FEM_EINVAL, "material %d out of range", mat);
    if (m->n_mat > 255) return fail(FEM_EINVAL, "k(T) tables need at most 255 materials");
    if (n < 0 || n > kKtMax) return fail(FEM_EINVAL, "a k(T) table has 0 to %d points", kKtMax);
    if (n > 0 && (!T || !k)) return fail(FEM_EINVAL, "NULL array argument");
    for (int32_t j = 0; j < n; j++) {
        if (!std::isfinite(T[j]) || !std::isfinite(k[j]) || !(k[j] > 0.0))
            return fail(FEM_EINVAL, "k(T) point %d: T finite and k > 0 required", j);
        if (j > 0 && !(T[j] > T[j - 1])) return fail(FEM_EINVAL, "k(T) points must have ascending T");
    }
    fem_status st = invalidate_plan(m);
    if (st) return st;
    m->kt_T[(size_t)mat].assign(T, T + n);
    m->kt_k[(size_t)mat].assign(k, k + n);
    m->has_kt = false;
    for (const auto &v : m->kt_T) m->has_kt |= !v.empty();
    return ok();
}

fem_status fem_set_interface(fem_mesh *m, const int32_t *faces_a, int64_t n_a, const double *h_a,
                             const int32_t *faces_b, int64_t n_b, const double *h_b)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (m->n_inst > 0) return fail(FEM_ESTATE, "a batch takes its materials and boundaries from its parts");
    if (n_a < 0 || n_b < 0 || (n_a > 0) != (n_b > 0))
        return fail(FEM_EINVAL, "an interface needs faces on both sides (or none)");
    if (n_a > 0 && (!faces_a || !faces_b || !h_a || !h_b)) return fail(FEM_EINVAL, "NULL array argument");
    if (n_a + n_b > INT32_MAX / 3) return fail(FEM_EINVAL, "too many interface faces");
    const int64_t n = n_a + n_b;
    std::vector<int32_t> fc((size_t)(3 * n));
    std::vector<double> fa((size_t)n), g((size_t)n);
    std::vector<int64_t> sis;
    try {
        for (int64_t f = 0; f < n; f++) {
            const int32_t *src = f < n_a ? faces_a + 3 * f : faces_b + 3 * (f - n_a);
            const double hh = f < n_a ? h_a[f] : h_b[f - n_a];
            for (int c = 0; c < 3; c++) {
                if (src[c] < 0 || src[c] >= m->N)
                    return fail(FEM_EINVAL, "interface face %lld: node id out of range", (long long)f);
                fc[3 * f + c] = src[c];
            }
            if (!std::isfinite(hh) || hh < 0)
                return fail(FEM_EINVAL, "interface face %lld: h must be finite and >= 0", (long long)f);
            const double *xa = &m->xyz[3 * (size_t)fc[3 * f]], *xb = &m->xyz[3 * (size_t)fc[3 * f + 1]],
                         *xc = &m->xyz[3 * (size_t)fc[3 * f + 2]];
            double u[3] = {xb[0] - xa[0], xb[1] - xa[1], xb[2] - xa[2]};
            double v[3] = {xc[0] - xa[0], xc[1] - xa[1], xc[2] - xa[2]};
            double nx = u[1] * v[2] - u[2] * v[1], ny = u[2] * v[0] - u[0] * v[2],
                   nz = u[0] * v[1] - u[1] * v[0];
            double A = 0.5 * std::sqrt(nx * nx + ny * ny + nz * nz);
            fa[f] = hh * A / 12.0;
            g[f] = A / 3.0 * hh;
        }
        std::vector<int32_t> owner;
        std::string err = face_owners(n, fc.data(), m->tets.data(), m->adj, owner);
        if (!err.empty()) return fail(FEM_EINVAL, "interface: %s", err.c_str());
        interface_sisters(m->xyz.data(), n_a, n_b, fc.data(), sis);
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    fem_status st = invalidate_plan(m);
    if (st) return st;
    m->if_faces.swap(fc);
    m->if_fa.swap(fa);
    m->if_g.swap(g);
    m->if_sister.swap(sis);
    m->F_if = n;
    combine_faces(m);
    return ok();
}

fem_status fem_set_dirichlet(fem_mesh *m, const int32_t *nodes, int64_t n, const double *T)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (n < 0 || (n > 0 && (!nodes || !T))) return fail(FEM_EINVAL, "bad Dirichlet arguments");
    if (m->n_inst > 0) return fail(FEM_ESTATE, "a batch takes its materials and boundaries from its parts");
    std::vector<uint8_t> is((size_t)m->N, 0);
    std::vector<double> val((size_t)m->N, 0.0);
    for (int64_t i = 0; i < n; i++) {
        if (nodes[i] < 0 || nodes[i] >= m->N) return fail(FEM_EINVAL, "Dirichlet node id out of range");
        if (!std::isfinite(T[i])) return fail(FEM_EINVAL, "non-finite Dirichlet temperature");
        is[nodes[i]] = 1;
        val[nodes[i]] = T[i];
    }
    fem_status st = invalidate_plan(m);
    if (st) return st;
    if (n == 0) {
        m->is_dir.clear();
        m->dir_T.clear();
    } else {
        m->is_dir.swap(is);
        m->dir_T.swap(val);
    }
    return ok();
}

fem_status fem_set_temperature(fem_mesh *m, const double *T0)
{
    if (!m || !T0) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    if (!finite_all(T0, m->N)) return fail(FEM_EINVAL, "non-finite initial temperature");
    m->pending.assign(T0, T0 + m->N);
    m->state = fem_mesh::ST_PENDING_T;
    m->step = 0;
    m->time = 0.0;
    m->q_carry = 0.0;
    m->acct_exact = true;
    m->acct_steps = 0;
    m->acct_T0max = *std::max_element(T0, T0 + m->N);
    m->env_U = -1.0;
    if (m->n_inst > 0) {
        m->inst_t.assign((size_t)m->n_inst, 0.0);
        m->inst_steps.assign((size_t)m->n_inst, 0);
    }
    if (m->dev_ok) {
        cudaSetDevice(m->device);
        fem_status st = m->prec == FEM_FP32 ? apply_pending<float>(m) : apply_pending<double>(m);
        if (st) return st;
    }
    return ok();
}

fem_status fem_set_state(fem_mesh *m, const double *E, int64_t step, double t)
{
    if (!m || !E) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    if (m->dev_ok && m->state == fem_mesh::ST_DEVICE) {
        // non-finite values are detected on the device and reported by the
        // next fem_get_* call
        // stage through the device buffer on the mesh's stream, no synchronisation
        cudaSetDevice(m->device);
        CU(cudaMemcpyAsync(m->dIo, E, (size_t)m->N * sizeof(double), cudaMemcpyHostToDevice, m->stream));
        KERNEL((m->prec == FEM_FP32 ? launch_upload<float, double>(m, m->dIo)
                                    : launch_upload<double, double>(m, m->dIo)),
               "state kernel");
    } else {
        if (!finite_all(E, m->N)) return fail(FEM_EINVAL, "non-finite enthalpy");
        m->pending.assign(E, E + m->N);
        m->state = fem_mesh::ST_PENDING_E;
        if (m->dev_ok) {
            cudaSetDevice(m->device);
            fem_status st = m->prec == FEM_FP32 ? apply_pending<float>(m) : apply_pending<double>(m);
            if (st) return st;
        }
    }
    m->step = step;
    m->time = t;
    m->acct_exact = false;   // the uploaded state need not balance the account
    return ok();
}

fem_status fem_set_allocator(fem_mesh *m, fem_alloc_fn alloc, fem_free_fn free_fn, void *ctx)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(FEM_EINVAL, "give both functions or neither");
    if (m->dev_ok) return fail(FEM_ESTATE, "the mesh already holds device memory");
    m->alloc_fn = alloc;
    m->free_fn = free_fn;
    m->alloc_ctx = ctx;
    return ok();
}

fem_status fem_set_stream(fem_mesh *m, void *cuda_stream)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    m->stream = (cudaStream_t)cuda_stream;
    return ok();
}

fem_status fem_stable_dt(fem_mesh *m, double *dt_out)
{
    if (!m || !dt_out) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    try {
        const std::vector<int32_t> sn = sister_nodes(m);
        const std::vector<double> wk = element_weights(m, true);
        *dt_out = gershgorin_dt(m->N, m->E, m->tets.data(), wk.data(), m->adj, m->F,
                                m->faces.data(), m->fa.data(), m->Cn.data(),
                                m->is_dir.empty() ? nullptr : m->is_dir.data(), m->F_if,
                                sn.data());
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    return ok();
}

fem_status fem_step(fem_mesh *m, int64_t n_steps, double dt)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (n_steps < 0) return fail(FEM_EINVAL, "n_steps must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(FEM_EINVAL, "dt must be positive and finite");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    if (m->state == fem_mesh::ST_NONE) return fail(FEM_ESTATE, "no initial state (call fem_set_temperature)");
    fem_status st = ready_for_io(m);
    if (st) return st;
    if (n_steps == 0) return ok();
    st = m->prec == FEM_FP32 ? step_impl<float>(m, n_steps, dt) : step_impl<double>(m, n_steps, dt);
    if (st) return st;
    for (int32_t i = 0; i < m->n_inst; i++) {
        m->inst_t[(size_t)i] += dt * (double)n_steps;
        m->inst_steps[(size_t)i] += n_steps;
    }
    return ok();
}

fem_status fem_step_profile(fem_mesh *m, int64_t n_steps, double dt, double *ms_out,
                            int32_t capacity, int32_t *n_used)
{
    if (!m || !ms_out || !n_used) return fail(FEM_EINVAL, "NULL argument");
    if (n_steps < 0) return fail(FEM_EINVAL, "n_steps must be >= 0");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(FEM_EINVAL, "dt must be positive and finite");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    if (m->state == fem_mesh::ST_NONE) return fail(FEM_ESTATE, "no initial state (call fem_set_temperature)");
    fem_status st = ready_for_io(m);
    if (st) return st;
    const int nk = step_kernel_count(m);
    if (capacity < nk) return fail(FEM_EINVAL, "capacity %d < %d kernels per step", capacity, nk);
    for (int k = 0; k < nk; k++) ms_out[k] = 0.0;
    *n_used = nk;
    st = m->prec == FEM_FP32 ? step_profile_impl<float>(m, n_steps, dt, ms_out)
                             : step_profile_impl<double>(m, n_steps, dt, ms_out);
    if (st) return st;
    for (int32_t i = 0; i < m->n_inst; i++) {   // as fem_step: every instance took them
        m->inst_t[(size_t)i] += dt * (double)n_steps;
        m->inst_steps[(size_t)i] += n_steps;
    }
    return ok();
}

fem_status fem_autotune(fem_mesh *m, const int32_t *block_elems, const int32_t *threads, int32_t n,
                        int32_t steps, double dt, int32_t *best_out, double *ms_out)
{
    if (!m || !block_elems || !best_out) return fail(FEM_EINVAL, "NULL argument");
    if (n < 1 || n > 64) return fail(FEM_EINVAL, "n = %d candidates (1..64)", n);
    if (steps < 1) return fail(FEM_EINVAL, "steps must be >= 1");
    if (!(dt > 0.0) || !std::isfinite(dt)) return fail(FEM_EINVAL, "dt must be positive and finite");
    for (int32_t i = 0; i < n; i++) {
        const int32_t th = threads ? threads[i] : 0;
        if (block_elems[i] < 64 || block_elems[i] > 12288)
            return fail(FEM_EINVAL, "candidate %d: block_elems %d outside 64..12288", i, block_elems[i]);
        if (th != 0 && th != 128 && th != 256 && th != 512 && th != 1024)
            return fail(FEM_EINVAL, "candidate %d: threads %d (0, 128, 256, 512 or 1024)", i, th);
    }
    if (!is_block(m)) return fail(FEM_ESTATE, "autotuning applies to the block variant");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    fem_status st = ready_for_io(m);
    if (st) return st;
    if ((st = check_device_flag(m))) return st;
    if ((st = fold_instance_heat(m))) return st;
    if ((st = stash_state(m))) return st;
    // what the timed steps change, put back afterwards
    const std::vector<double> E0 = m->pending;
    const int64_t step0 = m->step, acct0 = m->acct_steps;
    const double time0 = m->time, q0 = m->q_carry;
    const fem_options opt0 = m->opt;
    const std::vector<double> it0 = m->inst_t, iq0 = m->inst_q;
    const std::vector<int64_t> is0 = m->inst_steps;
    auto restore = [&](const fem_options &o) {
        m->opt = o;
        reset_partition(m, E0);
        m->step = step0;
        m->acct_steps = acct0;
        m->time = time0;
        m->q_carry = q0;
        m->inst_t = it0;
        m->inst_q = iq0;
        m->inst_steps = is0;
    };
    int32_t best = -1;
    double best_ms = 0.0;
    for (int32_t i = 0; i < n; i++) {
        fem_options o = opt0;
        o.block_elems = block_elems[i];
        o.threads = threads ? threads[i] : 0;
        restore(o);
        double ms = std::numeric_limits<double>::infinity();
        st = ready_for_io(m);
        if (st == FEM_OK)
            st = m->prec == FEM_FP32 ? time_steps<float>(m, steps, dt, &ms)
                                     : time_steps<double>(m, steps, dt, &ms);
        else if (st == FEM_EINVAL)
            st = FEM_OK;   // this partition does not fit (shared memory, local nodes)
        if (st) {
            std::string keep = g_err;
            restore(opt0);
            g_err = keep;
            return st;
        }
        if (ms_out) ms_out[i] = ms;
        if (std::isfinite(ms) && (best < 0 || ms < best_ms)) {
            best = i;
            best_ms = ms;
        }
    }
    fem_options o = opt0;
    if (best >= 0) {
        o.block_elems = block_elems[best];
        o.threads = threads ? threads[best] : 0;
    }
    restore(o);
    if ((st = ready_for_io(m))) return st;
    if (best < 0) return fail(FEM_EINVAL, "no candidate partition fits on this device");
    *best_out = best;
    return ok();
}

}  // extern "C"

namespace {

// Pipelined host I/O with the caller's arrays of element type io (double,
// or float for the _f32 calls); see fem.h.
template <typename io>
fem_status set_state_async_impl(fem_mesh *m, const io *E, int64_t step, double t)
{
    if (!m || !E) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    fem_status st = ready_for_io(m);
    if (st) return st;
    if ((st = ensure_async(m))) return st;
    const int i = m->in_idx;
    // the copy into staging buffer i waits for the last kernel that read it
    CU(cudaStreamWaitEvent(m->up_stream, m->ev_in_free[i], 0));
    CU(cudaMemcpyAsync(m->dIn[i], E, (size_t)m->N * sizeof(io), cudaMemcpyHostToDevice, m->up_stream));
    CU(cudaEventRecord(m->ev_in_ready[i], m->up_stream));
    CU(cudaStreamWaitEvent(m->stream, m->ev_in_ready[i], 0));
    if (sizeof(io) == 4) {
        const float *src = reinterpret_cast<const float *>(m->dIn[i]);
        KERNEL((m->prec == FEM_FP32 ? launch_upload<float, float>(m, src) : launch_upload<double, float>(m, src)),
               "state kernel");
    } else {
        KERNEL((m->prec == FEM_FP32 ? launch_upload<float, double>(m, m->dIn[i])
                                    : launch_upload<double, double>(m, m->dIn[i])),
               "state kernel");
    }
    CU(cudaEventRecord(m->ev_in_free[i], m->stream));
    m->in_idx = 1 - i;
    m->step = step;
    m->time = t;
    m->acct_exact = false;   // the uploaded state need not balance the account
    return ok();
}

template <typename io>
fem_status get_temperature_async_impl(fem_mesh *m, io *T_out)
{
    if (!m || !T_out) return fail(FEM_EINVAL, "NULL argument");
    fem_status st = ready_for_io(m);
    if (st) return st;
    if ((st = ensure_async(m))) return st;
    const int j = m->out_idx;
    // staging buffer j is rewritten once its previous copy to the host is done
    CU(cudaStreamWaitEvent(m->stream, m->ev_out_free[j], 0));
    if (sizeof(io) == 4) {
        float *dst = reinterpret_cast<float *>(m->dOutT[j]);
        KERNEL(m->prec == FEM_FP32
                   ? launch_get_temperature_f32<float>(view_of<float>(m), (const float *)m->dRanges, dst,
                                                       m->dNodeOld, m->N, m->dErr, m->stream)
                   : launch_get_temperature_f32<double>(view_of<double>(m), (const double *)m->dRanges, dst,
                                                        m->dNodeOld, m->N, m->dErr, m->stream),
               "read-back kernel");
    } else {
        KERNEL(m->prec == FEM_FP32
                   ? launch_get_temperature<float>(view_of<float>(m), (const float *)m->dC,
                                                   (const float *)m->dLc, m->dPh,
                                                   (const float *)m->dRanges, m->dOutT[j], m->dNodeOld,
                                                   m->N, m->dErr, m->stream)
                   : launch_get_temperature<double>(view_of<double>(m), (const double *)m->dC,
                                                    (const double *)m->dLc, m->dPh,
                                                    (const double *)m->dRanges, m->dOutT[j],
                                                    m->dNodeOld, m->N, m->dErr, m->stream),
               "read-back kernel");
    }
    CU(cudaEventRecord(m->ev_out_ready[j], m->stream));
    CU(cudaStreamWaitEvent(m->down_stream, m->ev_out_ready[j], 0));
    CU(cudaMemcpyAsync(T_out, m->dOutT[j], (size_t)m->N * sizeof(io), cudaMemcpyDeviceToHost,
                       m->down_stream));
    CU(cudaEventRecord(m->ev_out_free[j], m->down_stream));
    m->out_idx = 1 - j;
    return ok();
}

}  // namespace

extern "C" {

fem_status fem_set_state_async(fem_mesh *m, const double *E, int64_t step, double t)
{
    return set_state_async_impl<double>(m, E, step, t);
}

fem_status fem_set_state_async_f32(fem_mesh *m, const float *E, int64_t step, double t)
{
    return set_state_async_impl<float>(m, E, step, t);
}

fem_status fem_get_temperature_async(fem_mesh *m, double *T_out)
{
    return get_temperature_async_impl<double>(m, T_out);
}

fem_status fem_get_temperature_async_f32(fem_mesh *m, float *T_out)
{
    return get_temperature_async_impl<float>(m, T_out);
}

fem_status fem_sync(fem_mesh *m)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (!m->dev_ok) return ok();
    cudaSetDevice(m->device);
    if (m->async_ok) {
        CU(cudaStreamSynchronize(m->up_stream));
        CU(cudaStreamSynchronize(m->down_stream));
    }
    fem_status st = check_device_flag(m);   // synchronises the mesh's stream
    return st ? st : ok();
}

fem_status fem_get_temperature(fem_mesh *m, double *T_out)
{
    if (!m || !T_out) return fail(FEM_EINVAL, "NULL argument");
    fem_status st = ready_for_io(m);
    if (st) return st;
    // one synchronisation: the flag read after the copy also reports what
    // earlier asynchronous calls left on the device
    KERNEL(m->prec == FEM_FP32
               ? launch_get_temperature<float>(view_of<float>(m), (const float *)m->dC,
                                               (const float *)m->dLc, m->dPh,
                                               (const float *)m->dRanges, m->dIo, m->dNodeOld, m->N,
                                               m->dErr, m->stream)
               : launch_get_temperature<double>(view_of<double>(m), (const double *)m->dC,
                                                (const double *)m->dLc, m->dPh,
                                                (const double *)m->dRanges, m->dIo, m->dNodeOld,
                                                m->N, m->dErr, m->stream),
           "read-back kernel");
    CU(cudaMemcpyAsync(T_out, m->dIo, (size_t)m->N * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    if ((st = check_device_flag(m))) return st;   // synchronises
    return ok();
}

fem_status fem_get_state(fem_mesh *m, double *E_out, int64_t *step, double *t)
{
    if (!m || !E_out) return fail(FEM_EINVAL, "NULL argument");
    fem_status st = ready_for_io(m);
    if (st) return st;
    if ((st = check_device_flag(m))) return st;
    KERNEL(m->prec == FEM_FP32
               ? launch_get_state<float>(view_of<float>(m), m->dIo, m->dNodeOld, m->N, m->stream)
               : launch_get_state<double>(view_of<double>(m), m->dIo, m->dNodeOld, m->N, m->stream),
           "read-back kernel");
    CU(cudaMemcpyAsync(E_out, m->dIo, (size_t)m->N * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    if (step) *step = m->step;
    if (t) *t = m->time;
    return ok();
}

fem_status fem_get_enthalpy(fem_mesh *m, double *h_out)
{
    fem_status st = fem_get_state(m, h_out, nullptr, nullptr);
    if (st) return st;
    for (int64_t i = 0; i < m->N; i++) h_out[i] /= m->mn[i];
    return ok();
}

fem_status fem_get_energy(fem_mesh *m, double out[4])
{
    if (!m || !out) return fail(FEM_EINVAL, "NULL argument");
    fem_status st = ready_for_io(m);
    if (st) return st;
    if ((st = check_device_flag(m))) return st;
    // FP64 reductions of the current state (sum E, latent) and of the
    // per-CTA cumulative boundary heat
    KERNEL(m->prec == FEM_FP32 ? energy_snapshot<float>(m) : energy_snapshot<double>(m),
           "energy kernel");
    double r[3];
    CU(cudaMemcpyAsync(r, m->dOut, 3 * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    out[0] = r[0];
    out[1] = m->U0;
    out[2] = r[2] + m->q_carry;
    out[3] = r[1];
    if (!std::isfinite(r[0]))
        return fail(FEM_EUNSTABLE, "non-finite total enthalpy: dt above the stable limit?");
    // Energy balance: in the enthalpy formulation every step conserves
    // U - Q_b exactly (zero column sums of K^e), so without Dirichlet nodes
    // U - U0 - Q_b only collects rounding.  Each step rounds every E_i once,
    // by at most half an ulp (2^-24 |E_i| in FP32, 2^-53 in FP64), and the
    // E_i of a stable run are positive (E = 0 at 0 K), so rounding alone
    // stays below 2 u (steps + 16) U_max with u the unit roundoff and U_max
    // the largest total enthalpy of the run.  A run past the stability
    // limit grows an oscillating mode whose rounding errors scale with
    // sum |E_i| >> U: it crosses that bound while every value is still
    // finite.
    // The scale is the larger of |U0| and |U|, with |U| capped by the
    // envelope a stable run cannot leave (the boundary heat of a blown-up
    // run grows with it and would otherwise move the bound along).
    if (m->acct_exact && !is_lm(m) && !has_dirichlet(m)) {
        const double u = m->prec == FEM_FP32 ? 0x1p-24 : 0x1p-53;
        const double scale =
            std::max(std::fabs(out[1]), std::min(std::fabs(out[0]), enthalpy_envelope(m)));
        const double bound = 2.0 * u * (double)(m->acct_steps + 16) * scale;
        const double resid = out[0] - out[1] - out[2];
        if (!(std::fabs(resid) <= bound)) {
            char msg[256];
            snprintf(msg, sizeof msg,
                     "energy balance residual U - U0 - Q_b = %.6g J exceeds the rounding bound "
                     "%.6g J after %lld steps: dt above the stable limit?",
                     resid, bound, (long long)m->acct_steps);
            return fail(FEM_EUNSTABLE, msg);
        }
    }
    return ok();
}

fem_status fem_mesh_info(fem_mesh *m, fem_info *out)
{
    if (!m || !out) return fail(FEM_EINVAL, "NULL argument");
    fem_status st = ensure_plan(m);
    if (st) return st;
    std::memset(out, 0, sizeof(*out));
    out->n_nodes = m->N;
    out->n_tets = m->E;
    out->n_faces = m->F;
    out->bandwidth_input = m->bw_input;
    out->bandwidth_internal = mesh_bandwidth(m->E, m->tets.data(), node_new_of(m).data());
    if (is_block(m)) {
        out->n_blocks = (int64_t)m->bp.blocks.size();
        out->n_interior_nodes = m->bp.n_int;
        out->n_shared_nodes = m->bp.n_sh;
        out->n_shared_copies = m->bp.n_copies;
        out->n_sched_rounds = m->bp.n_rounds;
        out->max_block_elems = m->bp.max_ne;
    } else {
        out->n_colors = m->fp.n_colors;
    }
    out->device_bytes = (int64_t)m->dev_bytes;
    out->precision = m->prec;
    out->variant = m->opt.variant;
    out->threads = is_block(m) ? (m->dev_ok ? m->threads : m->opt.threads) : 256;
    out->reorder = m->reorder;
    out->ctas_per_sm = m->ctas_per_sm;
    out->smem_per_cta = (int32_t)m->smem_bytes;
    out->n_instances = m->n_inst;
    out->n_faces = m->F_rb;
    out->n_interface_faces = (int32_t)m->F_if;
    return ok();
}

fem_status fem_rcm_order(int64_t n_nodes, const int32_t *tets, int64_t n_tets, int32_t *perm_out,
                         int64_t *bw_before, int64_t *bw_after)
{
    if (n_nodes <= 0 || n_tets <= 0 || !tets || !perm_out) return fail(FEM_EINVAL, "bad arguments");
    for (int64_t i = 0; i < 4 * n_tets; i++)
        if (tets[i] < 0 || tets[i] >= n_nodes) return fail(FEM_EINVAL, "node id out of range");
    try {
        NodeElems adj;
        build_node_elems(n_nodes, n_tets, tets, adj);
        std::vector<int32_t> perm;
        rcm_order(n_nodes, n_tets, tets, adj, perm);
        std::memcpy(perm_out, perm.data(), (size_t)n_nodes * sizeof(int32_t));
        if (bw_before) *bw_before = mesh_bandwidth(n_tets, tets, nullptr);
        if (bw_after) *bw_after = mesh_bandwidth(n_tets, tets, perm.data());
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    return ok();
}

fem_status fem_plan_array(fem_mesh *m, int32_t which, const void **data, int64_t *count)
{
    if (!m || !data || !count) return fail(FEM_EINVAL, "NULL argument");
    fem_status st = ensure_plan(m);
    if (st) return st;
    const bool block = is_block(m);
    auto give = [&](const void *p, size_t n) {
        *data = p;
        *count = (int64_t)n;
        return ok();
    };
    switch (which) {
    case 0: return block ? give(m->bp.node_new.data(), m->bp.node_new.size())
                         : give(m->fp.node_new.data(), m->fp.node_new.size());
    case 2: return block ? give(m->bp.elem_order.data(), m->bp.elem_order.size())
                         : give(m->fp.elem_order.data(), m->fp.elem_order.size());
    case 3: return block ? give(m->bp.face_order.data(), m->bp.face_order.size())
                         : give(m->fp.face_order.data(), m->fp.face_order.size());
    default: break;
    }
    if (which == 15) {
        m->if_sister32.assign(m->if_sister.begin(), m->if_sister.end());
        return give(m->if_sister32.data(), m->if_sister32.size());
    }
    if (!block) return fail(FEM_EINVAL, "plan array %d exists only for the block variant", which);
    switch (which) {
    case 1: return give(m->blocks_flat.data(), m->blocks_flat.size());
    case 4: return give(m->bp.copy_node.data(), m->bp.copy_node.size());
    case 5: return give(m->bp.sh_ptr.data(), m->bp.sh_ptr.size());
    case 6: return give(m->bp.sh_copy.data(), m->bp.sh_copy.size());
    case 7: return give(m->bp.grp.data(), m->bp.grp.size());
    case 8: return give(m->bp.sched.data(), m->bp.sched.size());
    case 9: return give(m->bp.elem_nodes.data(), m->bp.elem_nodes.size());
    case 10: return give(m->bp.face_nodes.data(), m->bp.face_nodes.size());
    case 11: return give(m->bp.copy_pos.data(), m->bp.copy_pos.size());
    case 12: return give(m->bp.block_inst.data(), m->bp.block_inst.size());
    case 13: return give(m->bp.inst_block_start.data(), m->bp.inst_block_start.size());
    case 14: return give(m->bp.inst_order.data(), m->bp.inst_order.size());
    default: return fail(FEM_EINVAL, "unknown plan array %d", which);
    }
}

// ---------------------------------------------------------------------------
// Batches of independent instances
// ---------------------------------------------------------------------------

fem_status fem_batch_create(fem_mesh *const *parts, int32_t n_parts, fem_mesh **out)
{
    if (!out) return fail(FEM_EINVAL, "out is NULL");
    *out = nullptr;
    if (!parts || n_parts <= 0) return fail(FEM_EINVAL, "need at least one part");
    const fem_mesh *p0 = parts[0];
    for (int32_t i = 0; i < n_parts; i++) {
        const fem_mesh *p = parts[i];
        if (!p) return fail(FEM_EINVAL, "part %d is NULL", i);
        if (p->n_inst > 0) return fail(FEM_EINVAL, "part %d is itself a batch", i);
        if (!p->have_mat) return fail(FEM_ESTATE, "part %d: fem_set_materials has not been called", i);
        if (p->state != fem_mesh::ST_PENDING_T)
            return fail(FEM_ESTATE, "part %d: set an initial temperature and do not step it", i);
        if (p->prec != p0->prec) return fail(FEM_EINVAL, "part %d: precision differs from part 0", i);
        if (p->opt.variant != FEM_VARIANT_BLOCK)
            return fail(FEM_EINVAL, "part %d: batches use the block variant", i);
        if (p->opt.formulation != p0->opt.formulation)
            return fail(FEM_EINVAL, "part %d: formulation differs from part 0", i);
    }
    std::unique_ptr<fem_mesh> m;
    try {
        m.reset(new fem_mesh());
        m->prec = p0->prec;
        m->reorder = p0->reorder;
        m->opt = p0->opt;
        m->n_inst = n_parts;
        m->inst_node.assign(1, 0);
        m->inst_elem.assign(1, 0);
        for (int32_t i = 0; i < n_parts; i++) {
            m->inst_node.push_back(m->inst_node.back() + parts[i]->N);
            m->inst_elem.push_back(m->inst_elem.back() + parts[i]->E);
        }
        m->N = m->inst_node.back();
        m->E = m->inst_elem.back();
        int64_t F_all = 0;
        for (int32_t i = 0; i < n_parts; i++) F_all += parts[i]->F;
        if (m->N > INT32_MAX - 1 || m->E > INT32_MAX / 8 || F_all > INT32_MAX / 3)
            return fail(FEM_EINVAL, "batch too large for 32-bit ids");
        // distinct phase-change ranges over all parts
        std::vector<std::vector<uint8_t>> rmap((size_t)n_parts);
        for (int32_t i = 0; i < n_parts; i++) {
            const fem_mesh *p = parts[i];
            for (size_t r = 0; r < p->ranges.size() / 2; r++) {
                int found = -1;
                for (size_t q = 0; q < m->ranges.size() / 2; q++)
                    if (m->ranges[2 * q] == p->ranges[2 * r] && m->ranges[2 * q + 1] == p->ranges[2 * r + 1])
                        found = (int)q;
                if (found < 0) {
                    if ((int)(m->ranges.size() / 2) >= kMaxRanges)
                        return fail(FEM_EINVAL, "more than %d distinct phase-change ranges", kMaxRanges);
                    found = (int)(m->ranges.size() / 2);
                    m->ranges.push_back(p->ranges[2 * r]);
                    m->ranges.push_back(p->ranges[2 * r + 1]);
                }
                rmap[(size_t)i].push_back((uint8_t)found);
            }
        }
        bool any_dir = false;
        for (int32_t i = 0; i < n_parts; i++) any_dir |= !parts[i]->is_dir.empty();
        for (int32_t i = 0; i < n_parts; i++) {
            const fem_mesh *p = parts[i];
            const int32_t no = (int32_t)m->inst_node[(size_t)i];
            m->xyz.insert(m->xyz.end(), p->xyz.begin(), p->xyz.end());
            for (int32_t v : p->tets) m->tets.push_back(v + no);
            // materials: identical ones (same properties and k(T) table) are
            // merged, so that many parts of a few alloys stay few materials
            std::vector<int32_t> mmap((size_t)p->n_mat);
            for (int32_t q = 0; q < p->n_mat; q++) {
                const fem_material &a = p->mats[(size_t)q];
                int32_t found = -1;
                for (int32_t r = 0; r < m->n_mat && found < 0; r++) {
                    const fem_material &b = m->mats[(size_t)r];
                    if (a.rho == b.rho && a.c == b.c && a.k == b.k && a.latent == b.latent &&
                        a.T_solidus == b.T_solidus && a.T_liquidus == b.T_liquidus &&
                        p->kt_T[(size_t)q] == m->kt_T[(size_t)r] && p->kt_k[(size_t)q] == m->kt_k[(size_t)r])
                        found = r;
                }
                if (found < 0) {
                    found = m->n_mat++;
                    m->mats.push_back(a);
                    m->mat_k.push_back(p->mat_k[(size_t)q]);
                    m->kt_T.push_back(p->kt_T[(size_t)q]);
                    m->kt_k.push_back(p->kt_k[(size_t)q]);
                }
                mmap[(size_t)q] = found;
            }
            for (int32_t v : p->mat) m->mat.push_back(mmap[(size_t)v]);
            m->has_kt |= p->has_kt;
            m->vol.insert(m->vol.end(), p->vol.begin(), p->vol.end());
            for (int32_t r : p->rank) m->rank.push_back(r + no);
            m->w.insert(m->w.end(), p->w.begin(), p->w.end());
            m->Cn.insert(m->Cn.end(), p->Cn.begin(), p->Cn.end());
            m->mn.insert(m->mn.end(), p->mn.begin(), p->mn.end());
            m->Lcn.insert(m->Lcn.end(), p->Lcn.begin(), p->Lcn.end());
            for (uint8_t r : p->rng_id) m->rng_id.push_back(rmap[(size_t)i].empty() ? 0 : rmap[(size_t)i][r]);
            for (int32_t v : p->rb_faces) m->rb_faces.push_back(v + no);
            m->rb_fa.insert(m->rb_fa.end(), p->rb_fa.begin(), p->rb_fa.end());
            m->rb_fg.insert(m->rb_fg.end(), p->rb_fg.begin(), p->rb_fg.end());
            const int64_t io = (int64_t)m->if_fa.size();
            for (int32_t v : p->if_faces) m->if_faces.push_back(v + no);
            m->if_fa.insert(m->if_fa.end(), p->if_fa.begin(), p->if_fa.end());
            m->if_g.insert(m->if_g.end(), p->if_g.begin(), p->if_g.end());
            for (int64_t v : p->if_sister) m->if_sister.push_back(v + io);
            if (any_dir) {
                if (p->is_dir.empty()) {
                    m->is_dir.insert(m->is_dir.end(), (size_t)p->N, 0);
                    m->dir_T.insert(m->dir_T.end(), (size_t)p->N, 0.0);
                } else {
                    m->is_dir.insert(m->is_dir.end(), p->is_dir.begin(), p->is_dir.end());
                    m->dir_T.insert(m->dir_T.end(), p->dir_T.begin(), p->dir_T.end());
                }
            }
            m->pending.insert(m->pending.end(), p->pending.begin(), p->pending.end());
            m->bw_input = std::max(m->bw_input, p->bw_input);
            m->bw_rank = std::max(m->bw_rank, p->bw_rank);
            const std::vector<int32_t> sn = sister_nodes(p);
            const std::vector<double> wk = element_weights(p, true);
            const double dt = gershgorin_dt(p->N, p->E, p->tets.data(), wk.data(), p->adj, p->F,
                                            p->faces.data(), p->fa.data(), p->Cn.data(),
                                            p->is_dir.empty() ? nullptr : p->is_dir.data(),
                                            p->F_if, sn.data());
            m->inst_stable.push_back(dt);
        }
        if (m->ranges.empty()) { m->ranges.push_back(0.0); m->ranges.push_back(0.0); }
        if ((m->has_kt || is_lm(m.get())) && m->n_mat > 255)
            return fail(FEM_EINVAL, "k(T) tables and the apparent-capacity formulation need at most 255 "
                                    "distinct materials in a batch");
        m->F_rb = (int64_t)m->rb_fa.size();
        m->F_if = (int64_t)m->if_fa.size();
        combine_faces(m.get());
        build_node_elems(m->N, m->E, m->tets.data(), m->adj);
        m->have_mat = true;
        m->state = fem_mesh::ST_PENDING_T;
        m->acct_exact = true;
        m->acct_steps = 0;
        m->acct_T0max = *std::max_element(m->pending.begin(), m->pending.end());
        m->inst_dt.resize((size_t)n_parts);
        for (int32_t i = 0; i < n_parts; i++) m->inst_dt[(size_t)i] = 0.9 * m->inst_stable[(size_t)i];
        m->inst_t.assign((size_t)n_parts, 0.0);
        m->inst_steps.assign((size_t)n_parts, 0);
        m->inst_q.assign((size_t)n_parts, 0.0);
        // plan order: the instances that need the most steps first (smallest
        // stable step), so that with step sizes proportional to the stable
        // ones the instances still stepping are always a prefix of the plan
        m->inst_plan_order.resize((size_t)n_parts);
        for (int32_t i = 0; i < n_parts; i++) m->inst_plan_order[(size_t)i] = i;
        std::stable_sort(m->inst_plan_order.begin(), m->inst_plan_order.end(), [&](int32_t a, int32_t b) {
            return m->inst_stable[(size_t)a] < m->inst_stable[(size_t)b];
        });
    } catch (const std::bad_alloc &) {
        return fail(FEM_ENOMEM, "host allocation failed");
    }
    *out = m.release();
    return ok();
}

fem_status fem_instance_stable_dt(fem_mesh *m, double *dt_out)
{
    if (!m || !dt_out) return fail(FEM_EINVAL, "NULL argument");
    if (m->n_inst == 0) return fail(FEM_ESTATE, "not a batch");
    std::copy(m->inst_stable.begin(), m->inst_stable.end(), dt_out);
    return ok();
}

fem_status fem_set_instance_dt(fem_mesh *m, const double *dt)
{
    if (!m || !dt) return fail(FEM_EINVAL, "NULL argument");
    if (m->n_inst == 0) return fail(FEM_ESTATE, "not a batch");
    for (int32_t i = 0; i < m->n_inst; i++)
        if (!(dt[i] > 0.0) || !std::isfinite(dt[i]))
            return fail(FEM_EINVAL, "instance %d: dt must be positive and finite", i);
    m->inst_dt.assign(dt, dt + m->n_inst);
    return ok();
}

fem_status fem_get_instance_times(fem_mesh *m, double *t_out, int64_t *steps_out)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (m->n_inst == 0) return fail(FEM_ESTATE, "not a batch");
    if (t_out) std::copy(m->inst_t.begin(), m->inst_t.end(), t_out);
    if (steps_out) std::copy(m->inst_steps.begin(), m->inst_steps.end(), steps_out);
    return ok();
}

}  // extern "C"

namespace {

// One fem_advance: per plan position k the number of steps; every step
// launches the block and exchange kernels once per run of consecutive plan
// positions still stepping (a single run when the counts do not increase
// along the plan).
template <typename real>
fem_status advance_launches(fem_mesh *m, const std::vector<int64_t> &nk, cudaStream_t st)
{
    const BlockPlan &bp = m->bp;
    BlockArgs<real> a = block_args<real>(m);
    a.blk_dt = (const real *)m->dBlkDt;
    a.sh_dt = (const real *)m->dShDt;
    const int64_t K = (int64_t)nk.size();
    int64_t max_n = 0;
    for (int64_t v : nk) max_n = std::max(max_n, v);
    for (int64_t step = 0; step < max_n; step++) {
        if (m->F_if > 0) {
            fem_status fs = launch_interface_kernel<real>(m, st);
            if (fs) return fs;
        }
        for (int64_t k0 = 0; k0 < K;) {
            if (nk[(size_t)k0] <= step) { k0++; continue; }
            int64_t k1 = k0;
            while (k1 < K && nk[(size_t)k1] > step) k1++;
            a.b_first = bp.inst_block_start[(size_t)k0];
            a.b_count = bp.inst_block_start[(size_t)k1] - a.b_first;
            a.s_first = bp.inst_sh_start[(size_t)k0];
            a.s_end = bp.inst_sh_start[(size_t)k1];
            KERNEL(launch_block_kernel<real>(a, m->threads, m->smem_bytes, 0.0, st, m->has_kt,
                                             is_lm(m), m->wg),
                   "block kernel");
            KERNEL(launch_shared_update<real>(a, 0.0, st), "shared-node kernel");
            k0 = k1;
        }
    }
    return FEM_OK;
}

template <typename real>
fem_status advance_impl(fem_mesh *m, double t_end)
{
    const BlockPlan &bp = m->bp;
    const int32_t ni = m->n_inst;
    // steps and step sizes per instance: n_i equal steps of at most dt_i
    std::vector<int64_t> n((size_t)ni, 0);
    std::vector<double> dtp((size_t)ni, 0.0);
    for (int32_t i = 0; i < ni; i++) {
        const double span = t_end - m->inst_t[(size_t)i];
        if (!(span > 0.0)) continue;
        const double r = span / m->inst_dt[(size_t)i];
        int64_t c = (int64_t)std::ceil(r * (1.0 - 1e-12));
        if (c < 1) c = 1;
        n[(size_t)i] = c;
        dtp[(size_t)i] = span / (double)c;
    }
    // per-block and per-shared-node step sizes (only when they change)
    if (dtp != m->dt_uploaded) {
        std::vector<real> bdt(bp.blocks.size()), sdt((size_t)std::max<int64_t>(bp.n_sh, 1), real(0));
        for (size_t b = 0; b < bp.blocks.size(); b++) bdt[b] = (real)dtp[(size_t)bp.block_inst[b]];
        for (size_t k = 0; k < bp.inst_order.size(); k++) {
            const real d = (real)dtp[(size_t)bp.inst_order[k]];
            for (int64_t sidx = bp.inst_sh_start[k]; sidx < bp.inst_sh_start[k + 1]; sidx++)
                sdt[(size_t)sidx] = d;
        }
        CU(cudaMemcpyAsync(m->dBlkDt, bdt.data(), bdt.size() * sizeof(real), cudaMemcpyHostToDevice,
                           m->stream));
        CU(cudaMemcpyAsync(m->dShDt, sdt.data(), sdt.size() * sizeof(real), cudaMemcpyHostToDevice,
                           m->stream));
        CU(cudaStreamSynchronize(m->stream));
        m->dt_uploaded = dtp;
    }
    std::vector<int64_t> nk(bp.inst_order.size());
    for (size_t k = 0; k < nk.size(); k++) nk[k] = n[(size_t)bp.inst_order[k]];
    // the whole advance is one CUDA graph, rebuilt when the step pattern
    // changes; launched on the mesh's stream (or a stream of the library's
    // own when that is the legacy default stream, which cannot be captured)
    cudaStream_t st = m->stream;
    if (!st) {
        if (!m->own_stream) CU(cudaStreamCreate(&m->own_stream));
        st = m->own_stream;
    }
    if (!m->graph || nk != m->graph_key) {
        if (m->graph) cudaGraphExecDestroy(m->graph);
        m->graph = nullptr;
        m->graph_key.clear();
        cudaGraph_t g = nullptr;
        CU(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        fem_status fs = advance_launches<real>(m, nk, st);
        cudaError_t ce = cudaStreamEndCapture(st, &g);
        if (fs) {
            if (g) cudaGraphDestroy(g);
            return fs;
        }
        if (ce != cudaSuccess) return fail(FEM_ECUDA, "graph capture failed: %s", cudaGetErrorString(ce));
        ce = cudaGraphInstantiate(&m->graph, g, 0);
        cudaGraphDestroy(g);
        if (ce != cudaSuccess) {
            m->graph = nullptr;
            return fail(FEM_ECUDA, "graph instantiation failed: %s", cudaGetErrorString(ce));
        }
        m->graph_key = nk;
    }
    CU(cudaGraphLaunch(m->graph, st));
    if (st != m->stream) CU(cudaStreamSynchronize(st));
    int64_t max_n = 0;
    for (int32_t i = 0; i < ni; i++) {
        if (n[(size_t)i] == 0) continue;
        m->inst_t[(size_t)i] = t_end;
        m->inst_steps[(size_t)i] += n[(size_t)i];
        max_n = std::max(max_n, n[(size_t)i]);
    }
    m->step += max_n;
    m->acct_steps += max_n;
    m->time = std::max(m->time, t_end);
    return FEM_OK;
}

// T(E) of one node on the host (Eqs. 5, 11; the same piecewise-linear
// inverse the kernels use), for per-instance latent-heat sums.
double host_temperature(double E, double C, double Lc, double Ts, double Tl)
{
    if (Lc <= 0.0) return E / C;
    const double Es = C * Ts;
    if (E <= Es) return E / C;
    if (E >= C * Tl + Lc) return (E - Lc) / C;
    if (Tl <= Ts) return Ts;
    return Ts + (E - Es) * (Tl - Ts) / (C * (Tl - Ts) + Lc);
}

}  // namespace

extern "C" {

fem_status fem_advance(fem_mesh *m, double t_end)
{
    if (!m) return fail(FEM_EINVAL, "NULL mesh");
    if (m->n_inst == 0) return fail(FEM_ESTATE, "not a batch");
    if (!std::isfinite(t_end)) return fail(FEM_EINVAL, "t_end must be finite");
    fem_status st = ready_for_io(m);
    if (st) return st;
    st = m->prec == FEM_FP32 ? advance_impl<float>(m, t_end) : advance_impl<double>(m, t_end);
    return st ? st : ok();
}

fem_status fem_get_instance_energy(fem_mesh *m, int32_t inst, double out[4])
{
    if (!m || !out) return fail(FEM_EINVAL, "NULL argument");
    if (m->n_inst == 0) return fail(FEM_ESTATE, "not a batch");
    if (inst < 0 || inst >= m->n_inst) return fail(FEM_EINVAL, "instance %d out of range", inst);
    fem_status st = ready_for_io(m);
    if (st) return st;
    if ((st = check_device_flag(m))) return st;
    std::vector<double> E((size_t)m->N), q(m->bp.blocks.size());
    KERNEL(m->prec == FEM_FP32
               ? launch_get_state<float>(view_of<float>(m), m->dIo, m->dNodeOld, m->N, m->stream)
               : launch_get_state<double>(view_of<double>(m), m->dIo, m->dNodeOld, m->N, m->stream),
           "read-back kernel");
    CU(cudaMemcpyAsync(E.data(), m->dIo, E.size() * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaMemcpyAsync(q.data(), m->dQcum, q.size() * sizeof(double), cudaMemcpyDeviceToHost, m->stream));
    CU(cudaStreamSynchronize(m->stream));
    double U = 0.0, lat = 0.0, Qb = m->inst_q[(size_t)inst];
    for (int64_t nn = m->inst_node[(size_t)inst]; nn < m->inst_node[(size_t)inst + 1]; nn++) {
        const double e = E[(size_t)nn];
        U += e;
        if (m->Lcn[(size_t)nn] > 0.0) {
            const int r = m->rng_id[(size_t)nn];
            lat += e - m->Cn[(size_t)nn] * host_temperature(e, m->Cn[(size_t)nn], m->Lcn[(size_t)nn],
                                                              m->ranges[2 * (size_t)r],
                                                              m->ranges[2 * (size_t)r + 1]);
        }
    }
    for (size_t b = 0; b < q.size(); b++)
        if (m->bp.block_inst[b] == inst) Qb += q[b];
    out[0] = U;
    out[1] = m->inst_U0[(size_t)inst];
    out[2] = Qb;
    out[3] = lat;
    return ok();
}

}  // extern "C"

// ---- accessors of the learned surrogate (fem_surrogate.cu) ----------------

int fem::surrogate_mesh_view(::fem_mesh *m, SurrogateMeshView *v)
{
    if (!m || !v) return fail(FEM_EINVAL, "NULL argument");
    if (!m->have_mat) return fail(FEM_ESTATE, "fem_set_materials has not been called");
    fem_status st = ensure_plan(m);
    if (st) return st;
    *v = SurrogateMeshView{};
    v->N = m->N;
    v->E = m->E;
    v->xyz = m->xyz.data();
    v->tets = m->tets.data();
    v->w = m->w.data();
    v->C = m->Cn.data();
    v->Lc = m->Lcn.data();
    v->rng_id = m->rng_id.data();
    v->ranges = m->ranges.data();
    v->n_ranges = (int32_t)(m->ranges.size() / 2);
    v->F_rb = m->F_rb;
    v->rb_faces = m->rb_faces.data();
    v->rb_fa = m->rb_fa.data();
    v->rb_fg = m->rb_fg.data();
    v->n_inst = m->n_inst;
    v->inst_node = m->n_inst ? m->inst_node.data() : nullptr;
    v->inst_dt = m->n_inst ? m->inst_dt.data() : nullptr;
    v->prec = m->prec;
    v->variant = m->opt.variant;
    v->formulation = m->opt.formulation;
    v->has_kt = m->has_kt ? 1 : 0;
    v->has_dir = has_dirichlet(m) ? 1 : 0;
    v->F_if = m->F_if;
    v->node_new = is_block(m) ? m->bp.node_new.data() : nullptr;
    return FEM_OK;
}

int fem::surrogate_mesh_device(::fem_mesh *m, StateView<float> *v, void **stream, int *device)
{
    if (!m || !v) return fail(FEM_EINVAL, "NULL argument");
    if (m->prec != FEM_FP32 || !is_block(m) || is_lm(m))
        return fail(FEM_EINVAL, "the surrogate needs an FP32 block-variant mesh in the enthalpy formulation");
    fem_status st = ready_for_io(m);
    if (st) return st;
    *v = view_of<float>(m);
    if (stream) *stream = (void *)m->stream;
    if (device) *device = m->device;
    return FEM_OK;
}

int fem::surrogate_mesh_advanced(::fem_mesh *m, int64_t n_steps, double dt)
{
    if (!m) return fail(FEM_EINVAL, "NULL argument");
    KERNEL(refresh_mirror<float>(m), "mirror kernel");
    m->step += n_steps;
    m->acct_exact = false;
    if (m->n_inst > 0) {
        double t_max = m->time;
        for (int32_t i = 0; i < m->n_inst; i++) {
            m->inst_t[(size_t)i] += m->inst_dt[(size_t)i] * (double)n_steps;
            m->inst_steps[(size_t)i] += n_steps;
            t_max = std::max(t_max, m->inst_t[(size_t)i]);
        }
        m->time = t_max;
    } else {
        m->time += dt * (double)n_steps;
    }
    return FEM_OK;
}
