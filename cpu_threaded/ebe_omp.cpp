// Threaded CPU baseline of the explicit EBE enthalpy step (Sections 3, 4.1.2;
// Eqs. 4, 5, 9, 11, 14).  It is a comparison point for the GPU library, timed
// on the host's cores beside it: neither the product (which runs only on the
// GPU) nor the FP64 oracle (which stays plain and single-threaded).
//
// Layout: elements are coloured greedily so that no two elements of a colour
// share a node, then stored colour by colour (connectivity and the six
// off-diagonal conductances w_ab = -K^e_ab in structure-of-arrays form).  One
// step is: T(E) for every node; for each colour, a parallel loop over its
// elements that adds r_a = sum_b w_ab (T_b - T_a) into the node residual with
// plain stores (no atomics, no races); the Robin faces the same way (their
// own colouring); then E += dt R.  Every sum runs in a fixed order, so results
// do not depend on the thread count.
//
// Precision: FP64 or FP32 state and arithmetic (set-up in FP64).
#include <omp.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>

namespace {

struct Geometry {
  std::vector<double> C, Lc, Ts, Tl;  // per node: lumped capacity, latent capacity, range
  std::vector<uint8_t> dir;           // per node: held fixed (Eq. 3)
};

// Greedy colouring of items with `arity` node ids each: the lowest colour not
// used by an item already coloured that shares a node.  Returns the colour
// count, or -1 when more than 256 colours would be needed.
int greedy_colour(const int32_t* ids, int arity, int64_t n_items, int64_t n_nodes,
                  std::vector<int32_t>& colour) {
  std::vector<uint64_t> used(size_t(n_nodes) * 4, 0);  // 256 colour bits per node
  colour.assign(size_t(n_items), 0);
  int n_col = 0;
  for (int64_t e = 0; e < n_items; ++e) {
    uint64_t m[4] = {0, 0, 0, 0};
    for (int a = 0; a < arity; ++a)
      for (int w = 0; w < 4; ++w) m[w] |= used[size_t(ids[e * arity + a]) * 4 + w];
    int c = -1;
    for (int w = 0; w < 4 && c < 0; ++w)
      if (~m[w]) c = w * 64 + __builtin_ctzll(~m[w]);
    if (c < 0) return -1;
    colour[size_t(e)] = c;
    n_col = std::max(n_col, c + 1);
    for (int a = 0; a < arity; ++a) used[size_t(ids[e * arity + a]) * 4 + c / 64] |= 1ull << (c % 64);
  }
  return n_col;
}

// Items sorted by colour (stable): order[k] is the k-th item, start[c] the
// first position of colour c.
void colour_order(const std::vector<int32_t>& colour, int n_col, std::vector<int64_t>& order,
                  std::vector<int64_t>& start) {
  start.assign(size_t(n_col) + 1, 0);
  for (int32_t c : colour) start[size_t(c) + 1]++;
  for (int c = 0; c < n_col; ++c) start[size_t(c) + 1] += start[size_t(c)];
  std::vector<int64_t> pos(start.begin(), start.end() - 1);
  order.resize(colour.size());
  for (size_t e = 0; e < colour.size(); ++e) order[size_t(pos[size_t(colour[e])]++)] = int64_t(e);
}

}  // namespace

struct ebe_cpu_base {
  virtual ~ebe_cpu_base() = default;
  virtual void step(int64_t n, double dt) = 0;
  virtual void temperature(double* T) const = 0;
  virtual void energy(double* out) const = 0;
  int n_threads = 1, n_colours = 0, n_face_colours = 0;
};

template <class real>
struct EbeCpu : ebe_cpu_base {
  int64_t N = 0, E = 0, F = 0;
  std::vector<int32_t> conn[4];  // per element, colour-major
  std::vector<real> w[6];        // w01 w02 w03 w12 w13 w23
  std::vector<int64_t> col_start;
  std::vector<int32_t> fconn[3];
  std::vector<real> fa, fg;      // hA/12 and (A/3)(h T_inf - q)
  std::vector<int64_t> fcol_start;
  std::vector<real> En, C, Lc, Ts, Tl, T, R;
  std::vector<uint8_t> dir;

  real T_of(int64_t i) const {
    const real e = En[size_t(i)], c = C[size_t(i)], l = Lc[size_t(i)];
    if (l == real(0)) return e / c;
    const real es = c * Ts[size_t(i)];
    if (e <= es) return e / c;
    const real el = c * Tl[size_t(i)] + l;
    if (e >= el) return (e - l) / c;
    const real dT = Tl[size_t(i)] - Ts[size_t(i)];
    if (dT == real(0)) return Ts[size_t(i)];
    return Ts[size_t(i)] + (e - es) / (el - es) * dT;
  }

  void step(int64_t n, double dt_) override {
    const real dt = real(dt_);
    const int ncol = int(col_start.size()) - 1, nfcol = int(fcol_start.size()) - 1;
#pragma omp parallel num_threads(n_threads)
    for (int64_t s = 0; s < n; ++s) {
#pragma omp for schedule(static)
      for (int64_t i = 0; i < N; ++i) {
        T[size_t(i)] = T_of(i);
        R[size_t(i)] = real(0);
      }
      for (int c = 0; c < ncol; ++c) {
#pragma omp for schedule(static)
        for (int64_t e = col_start[size_t(c)]; e < col_start[size_t(c) + 1]; ++e) {
          const size_t k = size_t(e);
          const int32_t a = conn[0][k], b = conn[1][k], cc = conn[2][k], d = conn[3][k];
          const real ta = T[size_t(a)], tb = T[size_t(b)], tc = T[size_t(cc)], td = T[size_t(d)];
          const real f01 = w[0][k] * (tb - ta), f02 = w[1][k] * (tc - ta), f03 = w[2][k] * (td - ta);
          const real f12 = w[3][k] * (tc - tb), f13 = w[4][k] * (td - tb), f23 = w[5][k] * (td - tc);
          R[size_t(a)] += f01 + f02 + f03;
          R[size_t(b)] += f12 + f13 - f01;
          R[size_t(cc)] += f23 - f02 - f12;
          R[size_t(d)] += -f03 - f13 - f23;
        }
      }
      for (int c = 0; c < nfcol; ++c) {
#pragma omp for schedule(static)
        for (int64_t f = fcol_start[size_t(c)]; f < fcol_start[size_t(c) + 1]; ++f) {
          const size_t k = size_t(f);
          const int32_t a = fconn[0][k], b = fconn[1][k], cc = fconn[2][k];
          const real ta = T[size_t(a)], tb = T[size_t(b)], tc = T[size_t(cc)];
          const real s3 = ta + tb + tc;
          R[size_t(a)] += fg[k] - fa[k] * (s3 + ta);
          R[size_t(b)] += fg[k] - fa[k] * (s3 + tb);
          R[size_t(cc)] += fg[k] - fa[k] * (s3 + tc);
        }
      }
#pragma omp for schedule(static)
      for (int64_t i = 0; i < N; ++i)
        if (!dir[size_t(i)]) En[size_t(i)] += dt * R[size_t(i)];
    }
  }

  void temperature(double* out) const override {
    for (int64_t i = 0; i < N; ++i) out[i] = double(T_of(i));
  }

  void energy(double* out) const override {
    double u = 0.0;
    for (int64_t i = 0; i < N; ++i) u += double(En[size_t(i)]);
    out[0] = u;
  }
};

extern "C" {

// Builds the baseline for a mesh.  xyz [n_nodes][3] (m); tets [n_tets][4];
// mat [n_tets]; mats [n_mat][6] rows (rho, c, k, latent, Ts, Tl); faces
// [n_faces][3] Robin triangles with h, t_inf, q per face (q may be NULL);
// dir_nodes / dir_T Dirichlet data (n_dir may be 0); T0 [n_nodes].
// fp32 != 0 selects FP32 state and arithmetic.  n_threads <= 0 uses all.
// Returns NULL on invalid input (an index out of range, a degenerate tet,
// more than 256 colours).
void* ebe_cpu_create(const double* xyz, int64_t n_nodes, const int32_t* tets, int64_t n_tets,
                     const int32_t* mat, const double* mats, int32_t n_mat, const int32_t* faces,
                     int64_t n_faces, const double* h, const double* t_inf, const double* q,
                     const int32_t* dir_nodes, int64_t n_dir, const double* dir_T,
                     const double* T0, int fp32, int n_threads) {
  if (n_nodes <= 0 || n_tets <= 0 || n_faces < 0 || n_mat <= 0) return nullptr;
  for (int64_t i = 0; i < 4 * n_tets; ++i)
    if (tets[i] < 0 || tets[i] >= n_nodes) return nullptr;
  for (int64_t i = 0; i < 3 * n_faces; ++i)
    if (faces[i] < 0 || faces[i] >= n_nodes) return nullptr;
  for (int64_t e = 0; e < n_tets; ++e)
    if (mat[e] < 0 || mat[e] >= n_mat) return nullptr;

  // element geometry (FP64): gradients of the barycentric coordinates are the
  // rows of J^{-1}, J = [x1-x0 | x2-x0 | x3-x0]; K^e = k |V| grad N grad N^T
  std::vector<double> wd(size_t(n_tets) * 6);
  Geometry g;
  g.C.assign(size_t(n_nodes), 0.0);
  g.Lc.assign(size_t(n_nodes), 0.0);
  g.Ts.assign(size_t(n_nodes), 0.0);
  g.Tl.assign(size_t(n_nodes), 0.0);
  g.dir.assign(size_t(n_nodes), 0);
  for (int64_t e = 0; e < n_tets; ++e) {
    const int32_t* t = tets + 4 * e;
    double x[4][3];
    for (int a = 0; a < 4; ++a)
      for (int d = 0; d < 3; ++d) x[a][d] = xyz[3 * int64_t(t[a]) + d];
    double e1[3], e2[3], e3[3];
    for (int d = 0; d < 3; ++d) {
      e1[d] = x[1][d] - x[0][d];
      e2[d] = x[2][d] - x[0][d];
      e3[d] = x[3][d] - x[0][d];
    }
    auto cross = [](const double* u, const double* v, double* o) {
      o[0] = u[1] * v[2] - u[2] * v[1];
      o[1] = u[2] * v[0] - u[0] * v[2];
      o[2] = u[0] * v[1] - u[1] * v[0];
    };
    double g1[3], g2[3], g3[3];
    cross(e2, e3, g1);
    cross(e3, e1, g2);
    cross(e1, e2, g3);
    const double det = e1[0] * g1[0] + e1[1] * g1[1] + e1[2] * g1[2];
    double l2 = 0.0;
    for (int d = 0; d < 3; ++d) l2 += e1[d] * e1[d] + e2[d] * e2[d] + e3[d] * e3[d];
    const double ell = std::sqrt(l2 / 3.0);
    if (!(std::fabs(det) / 6.0 >= 1e-12 * ell * ell * ell)) return nullptr;
    double gr[4][3];
    for (int d = 0; d < 3; ++d) {
      gr[1][d] = g1[d] / det;
      gr[2][d] = g2[d] / det;
      gr[3][d] = g3[d] / det;
      gr[0][d] = -(gr[1][d] + gr[2][d] + gr[3][d]);
    }
    const double V = std::fabs(det) / 6.0;
    const double* m = mats + 6 * mat[e];
    const double kV = m[2] * V;
    static const int pa[6] = {0, 0, 0, 1, 1, 2}, pb[6] = {1, 2, 3, 2, 3, 3};
    for (int p = 0; p < 6; ++p) {
      const double* u = gr[pa[p]];
      const double* v = gr[pb[p]];
      wd[size_t(e) * 6 + size_t(p)] = -kV * (u[0] * v[0] + u[1] * v[1] + u[2] * v[2]);
    }
    for (int a = 0; a < 4; ++a) {
      g.C[size_t(t[a])] += m[0] * m[1] * V / 4.0;
      if (m[3] > 0.0) {
        g.Lc[size_t(t[a])] += m[0] * m[3] * V / 4.0;
        g.Ts[size_t(t[a])] = m[4];
        g.Tl[size_t(t[a])] = m[5];
      }
    }
  }
  for (int64_t i = 0; i < n_dir; ++i) {
    if (dir_nodes[i] < 0 || dir_nodes[i] >= n_nodes) return nullptr;
    g.dir[size_t(dir_nodes[i])] = 1;
  }

  std::vector<int32_t> colour;
  const int n_col = greedy_colour(tets, 4, n_tets, n_nodes, colour);
  std::vector<int32_t> fcolour;
  const int n_fcol = n_faces ? greedy_colour(faces, 3, n_faces, n_nodes, fcolour) : 0;
  if (n_col < 0 || n_fcol < 0) return nullptr;

  auto make = [&](auto tag) -> ebe_cpu_base* {
    using real = decltype(tag);
    auto* s = new EbeCpu<real>();
    s->N = n_nodes;
    s->E = n_tets;
    s->F = n_faces;
    s->n_threads = n_threads > 0 ? n_threads : omp_get_max_threads();
    s->n_colours = n_col;
    s->n_face_colours = n_fcol;
    std::vector<int64_t> order;
    colour_order(colour, n_col, order, s->col_start);
    for (int a = 0; a < 4; ++a) s->conn[a].resize(size_t(n_tets));
    for (int p = 0; p < 6; ++p) s->w[p].resize(size_t(n_tets));
    for (int64_t k = 0; k < n_tets; ++k) {
      const int64_t e = order[size_t(k)];
      for (int a = 0; a < 4; ++a) s->conn[a][size_t(k)] = tets[4 * e + a];
      for (int p = 0; p < 6; ++p) s->w[p][size_t(k)] = real(wd[size_t(e) * 6 + size_t(p)]);
    }
    if (n_faces) {
      colour_order(fcolour, n_fcol, order, s->fcol_start);
    } else {
      order.clear();
      s->fcol_start.assign(1, 0);
    }
    for (int a = 0; a < 3; ++a) s->fconn[a].resize(size_t(n_faces));
    s->fa.resize(size_t(n_faces));
    s->fg.resize(size_t(n_faces));
    for (int64_t k = 0; k < n_faces; ++k) {
      const int64_t f = order[size_t(k)];
      const int32_t* t = faces + 3 * f;
      double u[3], v[3], c[3];
      for (int d = 0; d < 3; ++d) {
        u[d] = xyz[3 * int64_t(t[1]) + d] - xyz[3 * int64_t(t[0]) + d];
        v[d] = xyz[3 * int64_t(t[2]) + d] - xyz[3 * int64_t(t[0]) + d];
      }
      c[0] = u[1] * v[2] - u[2] * v[1];
      c[1] = u[2] * v[0] - u[0] * v[2];
      c[2] = u[0] * v[1] - u[1] * v[0];
      const double A = 0.5 * std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
      for (int a = 0; a < 3; ++a) s->fconn[a][size_t(k)] = t[a];
      s->fa[size_t(k)] = real(h[f] * A / 12.0);
      s->fg[size_t(k)] = real(A / 3.0 * (h[f] * t_inf[f] - (q ? q[f] : 0.0)));
    }
    s->En.resize(size_t(n_nodes));
    s->C.resize(size_t(n_nodes));
    s->Lc.resize(size_t(n_nodes));
    s->Ts.resize(size_t(n_nodes));
    s->Tl.resize(size_t(n_nodes));
    s->T.assign(size_t(n_nodes), real(0));
    s->R.assign(size_t(n_nodes), real(0));
    s->dir = g.dir;
    std::vector<double> Td(T0, T0 + n_nodes);
    for (int64_t i = 0; i < n_dir; ++i) Td[size_t(dir_nodes[i])] = dir_T[i];
    for (int64_t i = 0; i < n_nodes; ++i) {
      const size_t j = size_t(i);
      double fl = 0.0;
      if (g.Lc[j] > 0.0) {
        if (g.Tl[j] > g.Ts[j])
          fl = std::min(1.0, std::max(0.0, (Td[j] - g.Ts[j]) / (g.Tl[j] - g.Ts[j])));
        else
          fl = Td[j] >= g.Ts[j] ? 1.0 : 0.0;
      }
      s->En[j] = real(g.C[j] * Td[j] + g.Lc[j] * fl);
      s->C[j] = real(g.C[j]);
      s->Lc[j] = real(g.Lc[j]);
      s->Ts[j] = real(g.Ts[j]);
      s->Tl[j] = real(g.Tl[j]);
    }
    return s;
  };
  return fp32 ? make(float(0)) : make(double(0));
}

void ebe_cpu_step(void* s, int64_t n_steps, double dt) {
  static_cast<ebe_cpu_base*>(s)->step(n_steps, dt);
}

void ebe_cpu_temperature(const void* s, double* T) {
  static_cast<const ebe_cpu_base*>(s)->temperature(T);
}

// out[0] = sum of the nodal enthalpies (J)
void ebe_cpu_energy(const void* s, double* out) {
  static_cast<const ebe_cpu_base*>(s)->energy(out);
}

// out[0] threads, out[1] element colours, out[2] face colours
void ebe_cpu_info(const void* s, int32_t* out) {
  const auto* b = static_cast<const ebe_cpu_base*>(s);
  out[0] = b->n_threads;
  out[1] = b->n_colours;
  out[2] = b->n_face_colours;
}

void ebe_cpu_destroy(void* s) { delete static_cast<ebe_cpu_base*>(s); }

}  // extern "C"
