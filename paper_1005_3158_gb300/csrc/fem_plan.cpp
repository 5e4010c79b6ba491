// Host-side preprocessing of libfem.  See fem_plan.h.
#include "fem_plan.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <functional>
#include <numeric>
#include <thread>

namespace fem {

namespace {

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

inline void sub3(const double *a, const double *b, double *o)
{
    o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2];
}
inline void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
inline double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// corner pair index used by the six stored conductances
constexpr int kPair[4][4] = {{-1, 0, 1, 2}, {0, -1, 3, 4}, {1, 3, -1, 5}, {2, 4, 5, -1}};

}  // namespace

void build_node_elems(int64_t N, int64_t E, const int32_t *tets, NodeElems &out)
{
    out.ptr.assign((size_t)N + 1, 0);
    for (int64_t i = 0; i < 4 * E; i++) out.ptr[(size_t)tets[i] + 1]++;
    for (int64_t n = 0; n < N; n++) out.ptr[n + 1] += out.ptr[n];
    out.elem.resize((size_t)(4 * E));
    std::vector<int64_t> fill(out.ptr.begin(), out.ptr.end() - 1);
    for (int64_t e = 0; e < E; e++)
        for (int c = 0; c < 4; c++) out.elem[fill[tets[4 * e + c]]++] = (int32_t)e;
}

double tet_signed_volume(const double *x0, const double *x1, const double *x2, const double *x3)
{
    double a[3], b[3], c[3], bc[3];
    sub3(x1, x0, a); sub3(x2, x0, b); sub3(x3, x0, c);
    cross3(b, c, bc);
    return dot3(a, bc) / 6.0;
}

void tet_conductances(const double *x0, const double *x1, const double *x2, const double *x3,
                      double k, double w[6], double *abs_vol)
{
    const double *x[4] = {x0, x1, x2, x3};
    double V = std::fabs(tet_signed_volume(x0, x1, x2, x3));
    double g[4][3];
    for (int a = 0; a < 4; a++) {
        // the face opposite corner a: corners j, k, l
        int j = (a + 1) & 3, kk = (a + 2) & 3, l = (a + 3) & 3;
        double u[3], v[3], n[3], d[3];
        sub3(x[kk], x[j], u);
        sub3(x[l], x[j], v);
        cross3(u, v, n);          // |n| = 2 * face area
        sub3(x[a], x[j], d);
        double s = dot3(n, d) > 0.0 ? 1.0 : -1.0;  // make n point towards a
        // grad N_a points into the tet towards a, |grad N_a| = area / (3V)
        for (int q = 0; q < 3; q++) g[a][q] = s * n[q] / (6.0 * V);
    }
    for (int a = 0; a < 4; a++)
        for (int b = a + 1; b < 4; b++) w[kPair[a][b]] = -k * V * dot3(g[a], g[b]);
    *abs_vol = V;
}

int64_t mesh_bandwidth(int64_t E, const int32_t *tets, const int32_t *perm)
{
    int64_t bw = 0;
    for (int64_t e = 0; e < E; e++) {
        int64_t lo = INT64_MAX, hi = INT64_MIN;
        for (int c = 0; c < 4; c++) {
            int64_t v = perm ? perm[tets[4 * e + c]] : tets[4 * e + c];
            lo = std::min(lo, v);
            hi = std::max(hi, v);
        }
        bw = std::max(bw, hi - lo);
    }
    return bw;
}

namespace {

// node graph (unique neighbours) as CSR
void node_graph(int64_t N, const int32_t *tets, const NodeElems &adj, std::vector<int64_t> &ptr,
                std::vector<int32_t> &nbr)
{
    std::vector<int32_t> mark((size_t)N, -1);
    ptr.assign((size_t)N + 1, 0);
    for (int64_t n = 0; n < N; n++) {
        int64_t d = 0;
        mark[n] = (int32_t)n;
        for (int64_t p = adj.ptr[n]; p < adj.ptr[n + 1]; p++) {
            int64_t e = adj.elem[p];
            for (int c = 0; c < 4; c++) {
                int32_t m = tets[4 * e + c];
                if (mark[m] != n) { mark[m] = (int32_t)n; d++; }
            }
        }
        ptr[n + 1] = ptr[n] + d;
    }
    nbr.resize((size_t)ptr[N]);
    std::fill(mark.begin(), mark.end(), -1);
    for (int64_t n = 0; n < N; n++) {
        int64_t q = ptr[n];
        mark[n] = (int32_t)n;
        for (int64_t p = adj.ptr[n]; p < adj.ptr[n + 1]; p++) {
            int64_t e = adj.elem[p];
            for (int c = 0; c < 4; c++) {
                int32_t m = tets[4 * e + c];
                if (mark[m] != n) { mark[m] = (int32_t)n; nbr[q++] = m; }
            }
        }
    }
}

// BFS from root over nodes with done[] == 0; returns the number of levels
// and the nodes of the last level.
int bfs_levels(int32_t root, const std::vector<int64_t> &ptr, const std::vector<int32_t> &nbr,
               const std::vector<uint8_t> &done, std::vector<int32_t> &stamp, int32_t tag,
               std::vector<int32_t> &queue, std::vector<int32_t> &last)
{
    queue.clear();
    queue.push_back(root);
    stamp[root] = tag;
    size_t head = 0;
    int levels = 0;
    while (head < queue.size()) {
        size_t end = queue.size();
        last.assign(queue.begin() + (int64_t)head, queue.begin() + (int64_t)end);
        levels++;
        for (; head < end; head++) {
            int32_t u = queue[head];
            for (int64_t p = ptr[u]; p < ptr[u + 1]; p++) {
                int32_t v = nbr[p];
                if (!done[v] && stamp[v] != tag) { stamp[v] = tag; queue.push_back(v); }
            }
        }
    }
    return levels;
}

}  // namespace

void rcm_order(int64_t N, int64_t E, const int32_t *tets, const NodeElems &adj,
               std::vector<int32_t> &perm)
{
    (void)E;
    std::vector<int64_t> ptr;
    std::vector<int32_t> nbr;
    node_graph(N, tets, adj, ptr, nbr);
    auto deg = [&](int32_t v) { return ptr[v + 1] - ptr[v]; };
    std::vector<uint8_t> done((size_t)N, 0);
    std::vector<int32_t> stamp((size_t)N, -1), queue, last, order, cand;
    order.reserve((size_t)N);
    int32_t tag = 0;
    for (int64_t seed = 0; seed < N; seed++) {
        if (done[seed]) continue;
        // pseudo-peripheral node of this component (George & Liu)
        int32_t r = (int32_t)seed;
        bfs_levels(r, ptr, nbr, done, stamp, ++tag, queue, last);
        // start from a minimum-degree node of the component
        for (int32_t v : queue)
            if (deg(v) < deg(r) || (deg(v) == deg(r) && v < r)) r = v;
        int ecc = bfs_levels(r, ptr, nbr, done, stamp, ++tag, queue, last);
        for (int it = 0; it < 8; it++) {
            int32_t c = last[0];
            for (int32_t v : last)
                if (deg(v) < deg(c) || (deg(v) == deg(c) && v < c)) c = v;
            int ecc_c = bfs_levels(c, ptr, nbr, done, stamp, ++tag, queue, last);
            if (ecc_c > ecc) { r = c; ecc = ecc_c; } else break;
        }
        // Cuthill-McKee from r: neighbours in ascending degree
        size_t head = order.size();
        order.push_back(r);
        done[r] = 1;
        while (head < order.size()) {
            int32_t u = order[head++];
            cand.clear();
            for (int64_t p = ptr[u]; p < ptr[u + 1]; p++) {
                int32_t v = nbr[p];
                if (!done[v]) { done[v] = 1; cand.push_back(v); }
            }
            std::sort(cand.begin(), cand.end(), [&](int32_t a, int32_t b) {
                return deg(a) != deg(b) ? deg(a) < deg(b) : a < b;
            });
            for (int32_t v : cand) order.push_back(v);
        }
    }
    perm.resize((size_t)N);
    for (int64_t i = 0; i < N; i++) perm[order[i]] = (int32_t)(N - 1 - i);
}

std::string face_owners(int64_t F, const int32_t *faces, const int32_t *tets,
                        const NodeElems &adj, std::vector<int32_t> &owner)
{
    owner.assign((size_t)F, -1);
    for (int64_t f = 0; f < F; f++) {
        int32_t a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
        if (a == b || b == c || a == c)
            return "face " + std::to_string(f) + " repeats a node";
        int count = 0;
        for (int64_t p = adj.ptr[a]; p < adj.ptr[a + 1]; p++) {
            int64_t e = adj.elem[p];
            bool hb = false, hc = false;
            for (int q = 0; q < 4; q++) {
                hb |= tets[4 * e + q] == b;
                hc |= tets[4 * e + q] == c;
            }
            if (hb && hc) { count++; owner[f] = (int32_t)e; }
        }
        if (count != 1)
            return "face " + std::to_string(f) + " is a face of " + std::to_string(count) +
                   " tets (a boundary face belongs to exactly one)";
    }
    return "";
}

int greedy_color(int64_t N, int64_t E, const int32_t *tets, const int32_t *order,
                 std::vector<int32_t> &color)
{
    constexpr int W = 4;  // up to 256 colours
    std::vector<uint64_t> used((size_t)N * W, 0);
    color.assign((size_t)E, -1);
    int ncol = 0;
    for (int64_t i = 0; i < E; i++) {
        int64_t e = order ? order[i] : i;
        uint64_t m[W] = {0, 0, 0, 0};
        for (int c = 0; c < 4; c++)
            for (int w = 0; w < W; w++) m[w] |= used[(size_t)tets[4 * e + c] * W + w];
        int col = -1;
        for (int w = 0; w < W && col < 0; w++)
            if (~m[w]) col = 64 * w + __builtin_ctzll(~m[w]);
        if (col < 0) return -1;
        color[e] = col;
        for (int c = 0; c < 4; c++)
            used[(size_t)tets[4 * e + c] * W + col / 64] |= 1ull << (col % 64);
        ncol = std::max(ncol, col + 1);
    }
    return ncol;
}

// ---------------------------------------------------------------------------
// Recursive coordinate bisection of element centroids
// ---------------------------------------------------------------------------
namespace {

struct Cen {
    float x[3];
    int32_t id;
};

// Splits a[0, n) into `parts` parts of balanced size: the first parts/2
// parts take the n*(parts/2)/parts items with the smallest coordinate along
// the longest axis of the bounding box, recursively.
void rcb(Cen *a, int64_t n, int64_t parts, int depth)
{
    if (parts <= 1) return;
    float lo[3] = {a[0].x[0], a[0].x[1], a[0].x[2]}, hi[3] = {lo[0], lo[1], lo[2]};
    for (int64_t i = 1; i < n; i++)
        for (int d = 0; d < 3; d++) {
            lo[d] = std::min(lo[d], a[i].x[d]);
            hi[d] = std::max(hi[d], a[i].x[d]);
        }
    int ax = 0;
    for (int d = 1; d < 3; d++)
        if (hi[d] - lo[d] > hi[ax] - lo[ax]) ax = d;
    int64_t p1 = parts / 2, p2 = parts - p1;
    int64_t mid = n * p1 / parts;
    std::nth_element(a, a + mid, a + n, [ax](const Cen &u, const Cen &v) {
        return u.x[ax] != v.x[ax] ? u.x[ax] < v.x[ax] : u.id < v.id;
    });
    if (depth < 3 && n > (1 << 20)) {
        std::thread t([=] { rcb(a, mid, p1, depth + 1); });
        rcb(a + mid, n - mid, p2, depth + 1);
        t.join();
    } else {
        rcb(a, mid, p1, depth + 1);
        rcb(a + mid, n - mid, p2, depth + 1);
    }
}

}  // namespace

namespace {

// Shared-memory bank cells of a slot: FP32 slots occupy one of 32 banks
// (one cell each); FP64 slots occupy a bank pair, of which 16 exist, and a
// warp access is two wavefronts, so each pair offers two cells.
struct BankModel {
    int real_size;
    int cells(uint32_t slot, int out[2]) const
    {
        if (real_size == 4) {
            out[0] = (int)(slot & 31u);
            return 1;
        }
        const int b = (int)(slot & 15u);
        out[0] = 2 * b;
        out[1] = 2 * b + 1;
        return 2;
    }
};

struct GroupMatcher {
    BankModel bm;
    int nrem[32];
    uint16_t rem[32][64];
    int owner[32];     // cell -> lane
    int choice[32];    // lane -> index into rem
    int choice_cell[32];

    bool augment(int l, uint32_t &seen)
    {
        for (int k = 0; k < nrem[l]; k++) {
            int cs[2];
            const int nc = bm.cells(rem[l][k], cs);
            for (int q = 0; q < nc; q++) {
                const int c = cs[q];
                if (seen & (1u << c)) continue;
                seen |= 1u << c;
                if (owner[c] < 0 || augment(owner[c], seen)) {
                    owner[c] = l;
                    choice[l] = k;
                    choice_cell[l] = c;
                    return true;
                }
            }
        }
        return false;
    }
};

// Reorders the slots of every row inside each 32-lane group (same number of
// rounds, same slots) so that each round's accesses fall into distinct
// bank cells where possible: a maximum lanes x cells matching per round,
// lanes that must advance to finish in time served first, the rest of
// those taking the least-loaded cell.  Rows change order only; the layout,
// the sizes and the slots of every node stay as planned.
void schedule_group(uint16_t *g, int J, uint16_t dummy, GroupMatcher &M)
{
    // g: J rounds in pairs: (round r, lane) at (r/2)*64 + 2*lane + r%2
    auto at = [&](int r, int lane) -> uint16_t & { return g[(r / 2) * 64 + 2 * lane + (r & 1)]; };
    for (int l = 0; l < 32; l++) {
        M.nrem[l] = 0;
        for (int r = 0; r < J; r++)
            if (at(r, l) != dummy) M.rem[l][M.nrem[l]++] = at(r, l);
    }
    for (int r = 0; r < J; r++) {
        const int left = J - r;
        int order[32], n = 0;
        for (int l = 0; l < 32; l++)
            if (M.nrem[l] > 0) order[n++] = l;
        std::sort(order, order + n, [&](int a, int b) { return M.nrem[a] > M.nrem[b]; });
        for (int c = 0; c < 32; c++) M.owner[c] = -1;
        for (int i = 0; i < n; i++) M.choice[order[i]] = -1;
        for (int i = 0; i < n; i++) {
            uint32_t seen = 0;
            M.augment(order[i], seen);
        }
        int load[32] = {0};
        for (int c = 0; c < 32; c++)
            if (M.owner[c] >= 0) load[c]++;
        // a lane that has as many slots left as rounds must take one now
        for (int i = 0; i < n; i++) {
            const int l = order[i];
            if (M.choice[l] >= 0 || M.nrem[l] < left) continue;
            int best = 0, best_load = 1 << 30;
            for (int k = 0; k < M.nrem[l]; k++) {
                int cs[2];
                const int nc = M.bm.cells(M.rem[l][k], cs);
                for (int q = 0; q < nc; q++)
                    if (load[cs[q]] < best_load) { best_load = load[cs[q]]; best = k; M.choice_cell[l] = cs[q]; }
            }
            M.choice[l] = best;
            load[M.choice_cell[l]]++;
        }
        for (int l = 0; l < 32; l++) {
            if (M.nrem[l] > 0 && M.choice[l] >= 0) {
                at(r, l) = M.rem[l][M.choice[l]];
                M.rem[l][M.choice[l]] = M.rem[l][--M.nrem[l]];
                M.choice[l] = -1;
            } else {
                at(r, l) = dummy;
            }
        }
    }
}

}  // namespace

void bank_schedule(BlockPlan &bp, int real_size)
{
    const int64_t nb = (int64_t)bp.blocks.size();
    unsigned nt = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    std::vector<std::thread> pool;
    for (unsigned t = 0; t < nt; t++)
        pool.emplace_back([&, t] {
            GroupMatcher M;
            M.bm.real_size = real_size;
            for (int64_t b = t; b < nb; b += nt) {
                const BlockInfo &bi = bp.blocks[(size_t)b];
                const uint16_t dummy = (uint16_t)(4 * bi.ne_pad + 3 * bi.nf_pad);
                for (int32_t gi = 0; gi < bi.ngrp; gi++) {
                    const int32_t r0 = bp.grp[(size_t)bi.g0 + gi], r1 = bp.grp[(size_t)bi.g0 + gi + 1];
                    if (r1 - r0 > 64) continue;   // rows longer than the matcher holds keep their order
                    schedule_group(bp.sched.data() + (size_t)r0 * 32, r1 - r0, dummy, M);
                }
            }
        });
    for (auto &th : pool) th.join();
}

std::string build_block_plan(int64_t N, int64_t E, const double *xyz, const int32_t *tets,
                             const std::vector<int32_t> &rank, int64_t F,
                             const int32_t *faces, const std::vector<int32_t> &face_owner,
                             int block_elems, int real_size, BlockPlan &out,
                             const std::vector<int64_t> &inst_elem_start,
                             const std::vector<int32_t> &inst_order)
{
    out = BlockPlan();
    out.N = N; out.E = E; out.F = F;
    // instances in plan order: element ranges [es[i], es[i+1]) of the caller
    std::vector<int64_t> es = inst_elem_start;
    std::vector<int32_t> order = inst_order;
    if (es.empty()) es = {0, E};
    const int64_t n_inst = (int64_t)es.size() - 1;
    if (order.empty())
        for (int64_t i = 0; i < n_inst; i++) order.push_back((int32_t)i);
    if ((int64_t)order.size() != n_inst || es[0] != 0 || es[(size_t)n_inst] != E)
        return "inconsistent instance ranges";
    // --- partition: element order and part starts; every instance is cut
    // into its own blocks (recursive coordinate bisection of the centroids),
    // instances one after another in plan order
    std::vector<Cen> cen((size_t)E);
    std::vector<int64_t> pstart;
    out.inst_order = order;
    out.inst_block_start.assign(1, 0);
    {
        int64_t off = 0;
        for (int64_t k = 0; k < n_inst; k++) {
            const int32_t i = order[(size_t)k];
            const int64_t e_lo = es[(size_t)i], n = es[(size_t)i + 1] - e_lo;
            if (n <= 0) return "instance " + std::to_string(i) + " has no elements";
            for (int64_t j = 0; j < n; j++) {
                const int64_t e = e_lo + j;
                double sc[3] = {0, 0, 0};
                for (int c = 0; c < 4; c++)
                    for (int d = 0; d < 3; d++) sc[d] += xyz[3 * (size_t)tets[4 * e + c] + d];
                for (int d = 0; d < 3; d++) cen[(size_t)(off + j)].x[d] = (float)(0.25 * sc[d]);
                cen[(size_t)(off + j)].id = (int32_t)e;
            }
            const int64_t parts = (n + block_elems - 1) / block_elems;
            rcb(cen.data() + off, n, parts, 0);
            // part starts follow from the same size recursion that rcb applies
            std::function<void(int64_t, int64_t, int64_t)> sizes =
                [&](int64_t o, int64_t m, int64_t pp) {
                    if (pp <= 1) { pstart.push_back(o); return; }
                    const int64_t p1 = pp / 2, mid = m * p1 / pp;
                    sizes(o, mid, p1);
                    sizes(o + mid, m - mid, pp - p1);
                };
            sizes(off, n, parts);
            for (int64_t q = 0; q < parts; q++) out.block_inst.push_back(i);
            out.inst_block_start.push_back((int32_t)pstart.size());
            off += n;
        }
    }
    const int64_t nparts = (int64_t)pstart.size();
    pstart.push_back(E);
    std::vector<int32_t> eorder((size_t)E);
    for (int64_t i = 0; i < E; i++) eorder[i] = cen[i].id;
    std::vector<Cen>().swap(cen);
    std::vector<int32_t> eblock((size_t)E);
    for (int64_t p = 0; p < nparts; p++)
        for (int64_t i = pstart[p]; i < pstart[p + 1]; i++) eblock[eorder[i]] = (int32_t)p;
    // --- faces grouped by the block of their owner element
    std::vector<int64_t> fcount((size_t)nparts + 1, 0);
    for (int64_t f = 0; f < F; f++) fcount[eblock[face_owner[f]] + 1]++;
    for (int64_t p = 0; p < nparts; p++) fcount[p + 1] += fcount[p];
    std::vector<int32_t> forder((size_t)F);
    {
        std::vector<int64_t> fill(fcount.begin(), fcount.end() - 1);
        for (int64_t f = 0; f < F; f++) forder[fill[eblock[face_owner[f]]]++] = (int32_t)f;
    }
    // --- node classification: number of distinct blocks touching each node
    std::vector<int32_t> nblk((size_t)N, 0), lastb((size_t)N, -1);
    for (int64_t p = 0; p < nparts; p++)
        for (int64_t i = pstart[p]; i < pstart[p + 1]; i++)
            for (int c = 0; c < 4; c++) {
                int32_t n = tets[4 * (size_t)eorder[i] + c];
                if (lastb[n] != p) { lastb[n] = (int32_t)p; nblk[n]++; }
            }
    for (int64_t n = 0; n < N; n++)
        if (nblk[n] == 0) return "node " + std::to_string(n) + " belongs to no tet";
    // signatures (sorted block lists) of shared nodes
    std::vector<int64_t> sig_ptr((size_t)N + 1, 0);
    for (int64_t n = 0; n < N; n++) sig_ptr[n + 1] = sig_ptr[n] + (nblk[n] > 1 ? nblk[n] : 0);
    std::vector<int32_t> sig((size_t)sig_ptr[N]);
    {
        std::vector<int64_t> fill(sig_ptr.begin(), sig_ptr.end() - 1);
        std::fill(lastb.begin(), lastb.end(), -1);
        for (int64_t p = 0; p < nparts; p++)
            for (int64_t i = pstart[p]; i < pstart[p + 1]; i++)
                for (int c = 0; c < 4; c++) {
                    int32_t n = tets[4 * (size_t)eorder[i] + c];
                    if (nblk[n] > 1 && lastb[n] != p) { lastb[n] = (int32_t)p; sig[fill[n]++] = (int32_t)p; }
                }
    }
    std::vector<int32_t> shared;
    for (int64_t n = 0; n < N; n++)
        if (nblk[n] > 1) shared.push_back((int32_t)n);
    std::sort(shared.begin(), shared.end(), [&](int32_t a, int32_t b) {
        int64_t la = sig_ptr[a + 1] - sig_ptr[a], lb = sig_ptr[b + 1] - sig_ptr[b];
        const int32_t *sa = &sig[sig_ptr[a]], *sb = &sig[sig_ptr[b]];
        for (int64_t k = 0; k < std::min(la, lb); k++)
            if (sa[k] != sb[k]) return sa[k] < sb[k];
        if (la != lb) return la < lb;
        return rank[a] < rank[b];
    });
    const int64_t n_sh = (int64_t)shared.size();
    const int64_t n_int = N - n_sh;
    // instances are independent: no node may be shared across two of them;
    // shared nodes sort by their first block, hence by plan position
    {
        std::vector<int32_t> bpos((size_t)nparts);
        for (int64_t k = 0; k < n_inst; k++)
            for (int32_t b = out.inst_block_start[(size_t)k]; b < out.inst_block_start[(size_t)k + 1]; b++)
                bpos[(size_t)b] = (int32_t)k;
        out.inst_sh_start.assign((size_t)n_inst + 1, n_sh);
        for (int64_t sidx = n_sh - 1; sidx >= 0; sidx--) {
            const int32_t n = shared[(size_t)sidx];
            const int32_t k = bpos[(size_t)sig[(size_t)sig_ptr[n]]];
            if (bpos[(size_t)sig[(size_t)sig_ptr[n + 1] - 1]] != k)
                return "node " + std::to_string(n) + " belongs to two instances";
            out.inst_sh_start[(size_t)k] = sidx;
        }
        for (int64_t k = n_inst - 1; k >= 0; k--)
            out.inst_sh_start[(size_t)k] = std::min(out.inst_sh_start[(size_t)k], out.inst_sh_start[(size_t)k + 1]);
    }
    std::vector<int32_t> sid((size_t)N, -1);
    for (int64_t s = 0; s < n_sh; s++) sid[shared[s]] = (int32_t)s;
    out.n_int = n_int; out.n_sh = n_sh;
    out.node_new.assign((size_t)N, -1);
    out.node_old.assign((size_t)N, -1);
    for (int64_t s = 0; s < n_sh; s++) {
        out.node_new[shared[s]] = (int32_t)(n_int + s);
        out.node_old[n_int + s] = shared[s];
    }
    // shared-node copy lists
    out.sh_ptr.assign((size_t)n_sh + 1, 0);
    for (int64_t s = 0; s < n_sh; s++) out.sh_ptr[s + 1] = out.sh_ptr[s] + nblk[shared[s]];
    out.n_copies = out.sh_ptr[n_sh];
    out.sh_copy.assign((size_t)out.n_copies, -1);
    out.copy_pos.assign((size_t)out.n_copies, -1);
    out.copy_node.assign((size_t)out.n_copies, -1);
    std::vector<int32_t> sh_fill(out.sh_ptr.begin(), out.sh_ptr.end() - 1);

    // --- per-block layout; every block's elements occupy the same stride
    // (the largest block rounded up to 8), so block b starts at b * nes
    int64_t nes = 8;
    for (int64_t p = 0; p < nparts; p++) nes = std::max(nes, round_up(pstart[p + 1] - pstart[p], 8));
    int64_t epos = 0, fpos = 0, cpos = 0, ipos = 0, rounds = 0, swords = 0;
    out.blocks.resize((size_t)nparts);
    std::vector<int32_t> loc((size_t)N, -1), cnt((size_t)N, 0);
    std::vector<int32_t> nodes_int, nodes_sh, row_ptr, rows, fillr;
    // elem_order / face_order / elem_nodes are sized at the end
    std::vector<int32_t> elem_order, face_order;
    elem_order.reserve((size_t)(E + 8 * nparts));
    face_order.reserve((size_t)(F + 8 * nparts));
    out.grp.reserve((size_t)(nparts * 40));
    for (int64_t p = 0; p < nparts; p++) {
        BlockInfo bi{};
        epos = p * nes;
        fpos = round_up(fpos, 8);
        elem_order.resize((size_t)epos, -1);
        face_order.resize((size_t)fpos, -1);
        bi.e0 = (int32_t)epos;
        bi.ne = (int32_t)(pstart[p + 1] - pstart[p]);
        bi.f0 = (int32_t)fpos;
        bi.nf = (int32_t)(fcount[p + 1] - fcount[p]);
        // corner rows of the slot array start 8 (FP32) or 4 (FP64) banks apart,
        // so the four corners of an element do not share a bank
        const int32_t corner_skew = real_size == 4 ? 8 : 4;
        bi.ne_pad = (int32_t)round_up(bi.ne, 32) + corner_skew;
        bi.nep = (int32_t)nes;
        bi.nf_pad = bi.nf ? (int32_t)round_up(bi.nf, 32) + corner_skew : 0;
        int64_t nslot = 4 * (int64_t)bi.ne_pad + 3 * (int64_t)bi.nf_pad;
        // slot nslot is the dummy target of schedule padding
        if (nslot + 1 > 65535)
            return "block " + std::to_string(p) + " needs " + std::to_string(nslot) +
                   " slots (> 65534); lower block_elems";
        const uint16_t dummy = (uint16_t)nslot;
        const int32_t *pe = &eorder[(size_t)pstart[p]];
        const int32_t *pf = &forder[(size_t)fcount[p]];
        // local nodes and their slot counts
        nodes_int.clear();
        nodes_sh.clear();
        for (int32_t i = 0; i < bi.ne; i++)
            for (int c = 0; c < 4; c++) {
                int32_t n = tets[4 * (size_t)pe[i] + c];
                if (cnt[n]++ == 0) (nblk[n] == 1 ? nodes_int : nodes_sh).push_back(n);
            }
        for (int32_t i = 0; i < bi.nf; i++)
            for (int c = 0; c < 3; c++) cnt[faces[3 * (size_t)pf[i] + c]]++;
        std::sort(nodes_int.begin(), nodes_int.end(), [&](int32_t a, int32_t b) {
            return cnt[a] != cnt[b] ? cnt[a] > cnt[b] : rank[a] < rank[b];
        });
        // shared copies by descending slot count too, so that the 32-lane
        // groups of the schedule hold rows of similar length (little
        // padding); ties keep the signature order
        std::sort(nodes_sh.begin(), nodes_sh.end(), [&](int32_t a, int32_t b) {
            return cnt[a] != cnt[b] ? cnt[a] > cnt[b] : sid[a] < sid[b];
        });
        bi.n0 = (int32_t)ipos;
        bi.nint = (int32_t)nodes_int.size();
        bi.c0 = (int32_t)cpos;
        bi.nsh = (int32_t)nodes_sh.size();
        for (int32_t k = 0; k < bi.nint; k++) {
            int32_t n = nodes_int[k];
            out.node_new[n] = (int32_t)(ipos + k);
            out.node_old[ipos + k] = n;
            loc[n] = k;
        }
        for (int32_t k = 0; k < bi.nsh; k++) {
            int32_t n = nodes_sh[k];
            loc[n] = bi.nint + k;
            out.copy_node[cpos + k] = (int32_t)(n_int + sid[n]);
            out.copy_pos[cpos + k] = sh_fill[sid[n]];
            out.sh_copy[sh_fill[sid[n]]++] = (int32_t)(cpos + k);
        }
        const int32_t nloc = bi.nint + bi.nsh;
        // rows: local node -> slots, elements first (block order), then faces
        row_ptr.assign((size_t)nloc + 1, 0);
        for (int32_t l = 0; l < nloc; l++) {
            int32_t n = l < bi.nint ? nodes_int[l] : nodes_sh[l - bi.nint];
            row_ptr[l + 1] = row_ptr[l] + cnt[n];
        }
        rows.assign((size_t)row_ptr[nloc], 0);
        fillr.assign(row_ptr.begin(), row_ptr.end() - 1);
        for (int32_t i = 0; i < bi.ne; i++)
            for (int c = 0; c < 4; c++) {
                int32_t l = loc[tets[4 * (size_t)pe[i] + c]];
                rows[fillr[l]++] = c * bi.ne_pad + i;
            }
        for (int32_t i = 0; i < bi.nf; i++)
            for (int c = 0; c < 3; c++) {
                int32_t l = loc[faces[3 * (size_t)pf[i] + c]];
                if (l < 0) return "face owner bookkeeping failed";
                rows[fillr[l]++] = 4 * bi.ne_pad + c * bi.nf_pad + i;
            }
        // 32-lane groups
        bi.g0 = (int32_t)out.grp.size();
        bi.r0 = (int32_t)rounds;
        bi.ngrp = (nloc + 31) / 32;
        for (int32_t g = 0; g < bi.ngrp; g++) {
            out.grp.push_back((int32_t)rounds);
            int32_t J = 0;
            for (int32_t lane = 0; lane < 32; lane++) {
                int32_t l = 32 * g + lane;
                if (l < nloc) J = std::max(J, row_ptr[l + 1] - row_ptr[l]);
            }
            J = (J + 1) & ~1;   // rounds go in pairs (one 32-bit word per lane)
            for (int32_t jp = 0; jp < J / 2; jp++)
                for (int32_t lane = 0; lane < 32; lane++)
                    for (int32_t h = 0; h < 2; h++) {
                        int32_t l = 32 * g + lane, j = 2 * jp + h;
                        uint16_t sl = dummy;
                        if (l < nloc && j < row_ptr[l + 1] - row_ptr[l])
                            sl = (uint16_t)rows[row_ptr[l] + j];
                        out.sched.push_back(sl);
                    }
            rounds += J;
        }
        out.grp.push_back((int32_t)rounds);
        bi.nrounds = (int32_t)(rounds - bi.r0);
        swords = std::max<int64_t>(swords, chunk_words(bi));   // the largest chunk
        // element / face positions
        for (int32_t i = 0; i < bi.ne; i++) elem_order.push_back(pe[i]);
        for (int32_t i = 0; i < bi.nf; i++) face_order.push_back(pf[i]);
        epos += bi.ne;
        fpos += bi.nf;
        ipos += bi.nint;
        cpos += bi.nsh;
        out.max_ne = std::max(out.max_ne, bi.ne);
        out.max_slots = std::max(out.max_slots, (size_t)nslot + 1);
        out.max_nloc = std::max(out.max_nloc, (size_t)nloc);
        // reset scratch
        for (int32_t n : nodes_int) { cnt[n] = 0; loc[n] = -1; }
        for (int32_t n : nodes_sh) { cnt[n] = 0; loc[n] = -1; }
        out.blocks[(size_t)p] = bi;
    }
    if (ipos != n_int || cpos != out.n_copies) return "node classification bookkeeping failed";
    // every block's schedule chunk sits at a fixed stride (the largest
    // chunk), so a CTA can copy it in before it has read its block header
    if (nparts * swords > INT32_MAX) return "schedule too large for 32-bit offsets";
    for (int64_t p = 0; p < nparts; p++) out.blocks[(size_t)p].s0 = (int32_t)(p * swords);
    out.chunk_stride = swords;
    out.n_sched_words = nparts * swords;
    out.E_pad = nparts * nes;
    out.F_pad = round_up(std::max<int64_t>(fpos, 1), 8);
    elem_order.resize((size_t)out.E_pad, -1);
    face_order.resize((size_t)out.F_pad, -1);
    out.elem_order.swap(elem_order);
    out.face_order.swap(face_order);
    out.n_rounds = rounds;
    out.elem_nodes.assign((size_t)out.E_pad * 4, -1);
    for (int64_t i = 0; i < out.E_pad; i++) {
        int32_t e = out.elem_order[i];
        if (e >= 0)
            for (int c = 0; c < 4; c++) out.elem_nodes[4 * i + c] = out.node_new[tets[4 * (size_t)e + c]];
    }
    out.face_nodes.assign((size_t)out.F_pad * 3, -1);
    for (int64_t i = 0; i < out.F_pad; i++) {
        int32_t f = out.face_order[i];
        if (f >= 0)
            for (int c = 0; c < 3; c++) out.face_nodes[3 * i + c] = out.node_new[faces[3 * (size_t)f + c]];
    }
    out.inst_int_start.assign((size_t)n_inst + 1, n_int);
    for (int64_t k = 0; k < n_inst; k++)
        out.inst_int_start[(size_t)k] = out.blocks[(size_t)out.inst_block_start[(size_t)k]].n0;
    bank_schedule(out, real_size);
    return "";
}

std::string build_flat_plan(int64_t N, int64_t E, const int32_t *tets,
                            const std::vector<int32_t> &rank, int64_t F, bool colored,
                            FlatPlan &out)
{
    out = FlatPlan();
    out.N = N; out.E = E; out.F = F;
    out.node_new = rank;
    out.node_old.assign((size_t)N, -1);
    for (int64_t n = 0; n < N; n++) out.node_old[rank[n]] = (int32_t)n;
    std::vector<int32_t> minnode((size_t)E);
    for (int64_t e = 0; e < E; e++) {
        int32_t m = INT32_MAX;
        for (int c = 0; c < 4; c++) m = std::min(m, rank[tets[4 * e + c]]);
        minnode[e] = m;
    }
    std::vector<int32_t> order((size_t)E);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(),
                     [&](int32_t a, int32_t b) { return minnode[a] < minnode[b]; });
    if (colored) {
        std::vector<int32_t> color;
        int nc = greedy_color(N, E, tets, order.data(), color);
        if (nc < 0) return "greedy colouring needs more than 256 colours";
        out.n_colors = nc;
        std::stable_sort(order.begin(), order.end(),
                         [&](int32_t a, int32_t b) { return color[a] < color[b]; });
        // colour classes start on 8-element boundaries
        out.color_start.assign((size_t)nc + 1, 0);
        std::vector<int32_t> padded;
        int64_t i = 0;
        for (int c = 0; c < nc; c++) {
            while (padded.size() % 8) padded.push_back(-1);
            out.color_start[c] = (int64_t)padded.size();
            while (i < E && color[order[i]] == c) padded.push_back(order[i++]);
        }
        while (padded.size() % 8 || padded.empty()) padded.push_back(-1);
        out.color_start[nc] = (int64_t)padded.size();
        out.elem_order.swap(padded);
    } else {
        out.elem_order = order;
        while (out.elem_order.size() % 8 || out.elem_order.empty()) out.elem_order.push_back(-1);
    }
    out.E_pad = (int64_t)out.elem_order.size();
    out.face_order.resize((size_t)F);
    std::iota(out.face_order.begin(), out.face_order.end(), 0);
    while (out.face_order.size() % 8 || out.face_order.empty()) out.face_order.push_back(-1);
    out.F_pad = (int64_t)out.face_order.size();
    return "";
}

double gershgorin_dt(int64_t N, int64_t E, const int32_t *tets, const double *w,
                     const NodeElems &adj, int64_t F, const int32_t *faces, const double *fa,
                     const double *C, const uint8_t *is_dir, int64_t F_if,
                     const int32_t *sister_nodes)
{
    (void)E;
    // node -> faces
    std::vector<int64_t> fptr((size_t)N + 1, 0);
    for (int64_t i = 0; i < 3 * F; i++) fptr[(size_t)faces[i] + 1]++;
    for (int64_t n = 0; n < N; n++) fptr[n + 1] += fptr[n];
    std::vector<int32_t> fidx((size_t)(3 * F));
    {
        std::vector<int64_t> fill(fptr.begin(), fptr.end() - 1);
        for (int64_t f = 0; f < F; f++)
            for (int c = 0; c < 3; c++) fidx[fill[faces[3 * f + c]]++] = (int32_t)f;
    }
    double lam = 0.0;
    std::vector<int32_t> col;
    std::vector<double> val;
    auto add = [&](int32_t j, double v) {
        for (size_t q = 0; q < col.size(); q++)
            if (col[q] == j) { val[q] += v; return; }
        col.push_back(j);
        val.push_back(v);
    };
    for (int64_t i = 0; i < N; i++) {
        if (is_dir && is_dir[i]) continue;
        col.clear();
        val.clear();
        for (int64_t p = adj.ptr[i]; p < adj.ptr[i + 1]; p++) {
            int64_t e = adj.elem[p];
            int a = 0;
            while (tets[4 * e + a] != i) a++;
            for (int b = 0; b < 4; b++) {
                if (b == a) continue;
                double wab = w[6 * e + kPair[a][b]];
                add((int32_t)i, wab);                 // K_ii = sum_b w_ab
                add(tets[4 * e + b], -wab);           // K_ij = -w_ab
            }
        }
        for (int64_t p = fptr[i]; p < fptr[i + 1]; p++) {
            int64_t f = fidx[p];
            for (int c = 0; c < 3; c++) {
                int32_t j = faces[3 * f + c];
                add(j, j == i ? 2.0 * fa[f] : fa[f]);
            }
            // an interface face also couples to its sister's nodes through
            // the ambient temperature: -h A / 9 = -(4/3) fa per pair
            const int64_t fi = f - (F - F_if);
            if (fi >= 0)
                for (int c = 0; c < 3; c++) add(sister_nodes[3 * fi + c], -4.0 / 3.0 * fa[f]);
        }
        double s = 0.0;
        for (double v : val) s += std::fabs(v);
        lam = std::max(lam, s / C[i]);
    }
    return lam > 0.0 ? 2.0 / lam : INFINITY;
}

void interface_sisters(const double *xyz, int64_t n_a, int64_t n_b, const int32_t *faces,
                       std::vector<int64_t> &sister)
{
    const int64_t n = n_a + n_b;
    sister.assign((size_t)n, -1);
    if (n_a == 0 || n_b == 0) return;
    std::vector<double> cen((size_t)(3 * n));
    for (int64_t f = 0; f < n; f++) {
        const double *x0 = xyz + 3 * (size_t)faces[3 * f], *x1 = xyz + 3 * (size_t)faces[3 * f + 1],
                     *x2 = xyz + 3 * (size_t)faces[3 * f + 2];
        for (int d = 0; d < 3; d++) cen[3 * f + d] = (x0[d] + x1[d] + x2[d]) / 3.0;
    }
    // one uniform grid per side over its centroids; a query scans rings of
    // cells around its own cell until no unscanned cell can be nearer
    struct Grid {
        double lo[3], h;
        int64_t n[3];
        std::vector<int64_t> ptr, idx;
    };
    auto build = [&](int64_t f0, int64_t cnt, Grid &g) {
        double hi[3];
        for (int d = 0; d < 3; d++) g.lo[d] = hi[d] = cen[3 * f0 + d];
        for (int64_t f = f0; f < f0 + cnt; f++)
            for (int d = 0; d < 3; d++) {
                g.lo[d] = std::min(g.lo[d], cen[3 * f + d]);
                hi[d] = std::max(hi[d], cen[3 * f + d]);
            }
        double ext = 0.0;
        for (int d = 0; d < 3; d++) ext = std::max(ext, hi[d] - g.lo[d]);
        // about two centroids per occupied cell of a surface
        g.h = std::max(ext / std::max(1.0, std::sqrt((double)cnt / 2.0)), 1e-30);
        for (;;) {   // at most ~8 cells per centroid
            for (int d = 0; d < 3; d++) g.n[d] = (int64_t)std::floor((hi[d] - g.lo[d]) / g.h) + 1;
            if ((double)g.n[0] * (double)g.n[1] * (double)g.n[2] <= 8.0 * (double)cnt + 64.0) break;
            g.h *= 1.5;
        }
        const int64_t cells = g.n[0] * g.n[1] * g.n[2];
        g.ptr.assign((size_t)cells + 1, 0);
        auto cell_of = [&](int64_t f) {
            int64_t c[3];
            for (int d = 0; d < 3; d++)
                c[d] = std::min(g.n[d] - 1, (int64_t)std::floor((cen[3 * f + d] - g.lo[d]) / g.h));
            return c[0] + g.n[0] * (c[1] + g.n[1] * c[2]);
        };
        for (int64_t f = f0; f < f0 + cnt; f++) g.ptr[(size_t)cell_of(f) + 1]++;
        for (int64_t c = 0; c < cells; c++) g.ptr[c + 1] += g.ptr[c];
        g.idx.assign((size_t)cnt, 0);
        std::vector<int64_t> fill(g.ptr.begin(), g.ptr.end() - 1);
        for (int64_t f = f0; f < f0 + cnt; f++) g.idx[(size_t)fill[(size_t)cell_of(f)]++] = f;
    };
    Grid ga, gb;
    build(0, n_a, ga);
    build(n_a, n_b, gb);
    for (int64_t f = 0; f < n; f++) {
        const Grid &g = f < n_a ? gb : ga;
        int64_t c[3];
        for (int d = 0; d < 3; d++)
            c[d] = std::max<int64_t>(0, std::min(g.n[d] - 1,
                                                 (int64_t)std::floor((cen[3 * f + d] - g.lo[d]) / g.h)));
        int64_t best = -1;
        double bd = 0.0;
        const int64_t rmax = std::max(g.n[0], std::max(g.n[1], g.n[2]));
        for (int64_t r = 0; r <= rmax; r++) {
            // every cell at Chebyshev distance r from c
            for (int64_t k = c[2] - r; k <= c[2] + r; k++)
                for (int64_t j = c[1] - r; j <= c[1] + r; j++)
                    for (int64_t i = c[0] - r; i <= c[0] + r; i++) {
                        if (std::max(std::abs(i - c[0]), std::max(std::abs(j - c[1]), std::abs(k - c[2]))) != r)
                            continue;
                        if (i < 0 || j < 0 || k < 0 || i >= g.n[0] || j >= g.n[1] || k >= g.n[2]) continue;
                        const int64_t cell = i + g.n[0] * (j + g.n[1] * k);
                        for (int64_t q = g.ptr[(size_t)cell]; q < g.ptr[(size_t)cell + 1]; q++) {
                            const int64_t o = g.idx[(size_t)q];
                            const double dx = cen[3 * o] - cen[3 * f], dy = cen[3 * o + 1] - cen[3 * f + 1],
                                         dz = cen[3 * o + 2] - cen[3 * f + 2];
                            const double dd = dx * dx + dy * dy + dz * dz;
                            if (best < 0 || dd < bd || (dd == bd && o < best)) { best = o; bd = dd; }
                        }
                    }
            // cells beyond ring r are at least r * h away from the query
            if (best >= 0 && (double)r * g.h > 0.0 && ((double)r * g.h) * ((double)r * g.h) > bd) break;
        }
        sister[(size_t)f] = best;
    }
}

}  // namespace fem
