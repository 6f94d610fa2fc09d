// Graph handle: CSR adjacency, normalised weights of D^-1/2 A D^-1/2 (Eq. gcn) and the
// nested bond neighbourhoods that bound the rows an exchange of s_i, s_j can change at
// each GCN layer.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <set>
#include <utility>
#include <vector>

#include "common.cuh"

namespace gna {

namespace {

struct HostGraph {
  int n = 0, E = 0, Lmax = 0;
  std::vector<int> row_ptr, col, col_edge, edges;
  std::vector<float> wf;
  std::vector<double> wd, J, Jz, hz, cb;
  std::vector<int> ball_off, ball_size, ball_vert, row_nbr, nbr_pos, max_ball, max_span;
  std::vector<int> ball_span, row_pack, bond_ent;  // compact forms, see DevGraph
  std::vector<int16_t> nbr_pos16;
  bool pack_ok = true;
};

gna_status validate(int32_t n_sites, int32_t n_edges, const int32_t* edges, const double* J,
                    int32_t max_layers, bool need_J) {
  if (n_sites < 1 || n_sites > 4096) return GNA_ERR_INVALID_ARG;
  if (n_edges < 0 || n_edges > (1 << 20)) return GNA_ERR_INVALID_ARG;
  if (max_layers < 0 || max_layers > kMaxL) return GNA_ERR_INVALID_ARG;
  if (n_edges > 0 && edges == nullptr) return GNA_ERR_INVALID_ARG;
  if (need_J && n_edges > 0 && J == nullptr) return GNA_ERR_INVALID_ARG;
  std::set<std::pair<int, int>> seen;
  for (int e = 0; e < n_edges; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    if (a < 0 || a >= n_sites || b < 0 || b >= n_sites || a == b) return GNA_ERR_INVALID_ARG;
    auto key = std::make_pair(a < b ? a : b, a < b ? b : a);
    if (!seen.insert(key).second) return GNA_ERR_INVALID_ARG;
    if (need_J && !std::isfinite(J[e])) return GNA_ERR_INVALID_ARG;
  }
  return GNA_OK;
}

void build(int n, int E, const int32_t* edges, const double* J, int Lmax, HostGraph* h) {
  h->n = n;
  h->E = E;
  h->Lmax = Lmax;
  std::vector<int> deg(n, 0);
  for (int e = 0; e < E; ++e) {
    deg[edges[2 * e]]++;
    deg[edges[2 * e + 1]]++;
  }
  h->row_ptr.assign(n + 1, 0);
  for (int v = 0; v < n; ++v) h->row_ptr[v + 1] = h->row_ptr[v] + deg[v];
  h->col.assign(2 * E, 0);
  h->col_edge.assign(2 * E, 0);
  std::vector<int> fill(h->row_ptr.begin(), h->row_ptr.end() - 1);
  // neighbours in edge-list order
  for (int e = 0; e < E; ++e) {
    int a = edges[2 * e], b = edges[2 * e + 1];
    h->col_edge[fill[a]] = e;
    h->col[fill[a]++] = b;
    h->col_edge[fill[b]] = e;
    h->col[fill[b]++] = a;
  }
  h->wf.resize(2 * E);
  h->wd.resize(2 * E);
  for (int v = 0; v < n; ++v)
    for (int k = h->row_ptr[v]; k < h->row_ptr[v + 1]; ++k) {
      double w = 1.0 / std::sqrt((double)deg[v] * (double)deg[h->col[k]]);
      h->wd[k] = w;
      h->wf[k] = (float)w;
    }
  h->edges.assign(edges, edges + 2 * E);
  if (J)
    h->J.assign(J, J + E);
  else
    h->J.assign(E, 1.0);

  // Nested neighbourhoods: ball_0 = (i, j); ball_l = ball_{l-1} followed by the
  // neighbours of its newest rows, in order of discovery.
  h->ball_off.assign(E + 1, 0);
  h->ball_size.assign((size_t)E * (Lmax + 1), 0);
  h->ball_span.assign((size_t)E * (Lmax + 1), 0);
  h->bond_ent.assign(E, 0);
  h->max_ball.assign(Lmax + 1, 0);
  h->max_span.assign(Lmax + 1, 0);
  h->ball_vert.clear();
  h->row_nbr.clear();
  h->nbr_pos.clear();
  std::vector<int> pos(n, -1), order;
  for (int e = 0; e < E; ++e) {
    order.clear();
    order.push_back(edges[2 * e]);
    order.push_back(edges[2 * e + 1]);
    pos[order[0]] = 0;
    pos[order[1]] = 1;
    int* sz = &h->ball_size[(size_t)e * (Lmax + 1)];
    sz[0] = 2;
    int lo = 0;
    for (int l = 1; l <= Lmax; ++l) {
      int hi = (int)order.size();
      for (int r = lo; r < hi; ++r) {
        int v = order[r];
        for (int k = h->row_ptr[v]; k < h->row_ptr[v + 1]; ++k) {
          int u = h->col[k];
          if (pos[u] < 0) {
            pos[u] = (int)order.size();
            order.push_back(u);
          }
        }
      }
      lo = hi;
      sz[l] = (int)order.size();
    }
    for (int l = 0; l <= Lmax; ++l) {
      if (sz[l] > h->max_ball[l]) h->max_ball[l] = sz[l];
      int span = 0;
      for (int r = 0; r < sz[l]; ++r) span += h->row_ptr[order[r] + 1] - h->row_ptr[order[r]];
      if (span > h->max_span[l]) h->max_span[l] = span;
      h->ball_span[(size_t)e * (Lmax + 1) + l] = span;
    }
    h->ball_off[e] = (int)h->ball_vert.size();
    h->bond_ent[e] = (int)h->nbr_pos.size();
    for (int r = 0; r < (int)order.size(); ++r) {
      int v = order[r];
      const int start = (int)h->nbr_pos.size() - h->bond_ent[e];
      if (start > 0xFFFF) h->pack_ok = false;
      h->ball_vert.push_back(v);
      h->row_nbr.push_back((int)h->nbr_pos.size());
      h->row_pack.push_back(v | ((start & 0xFFFF) << 16));
      for (int k = h->row_ptr[v]; k < h->row_ptr[v + 1]; ++k) {
        int u = h->col[k];
        h->nbr_pos.push_back(pos[u] >= 0 ? pos[u] : INT_MAX);
        h->nbr_pos16.push_back((int16_t)(pos[u] >= 0 ? pos[u] : 32767));
      }
    }
    for (int v : order) pos[v] = -1;
  }
  h->ball_off[E] = (int)h->ball_vert.size();
}

template <typename T>
gna_status upload(gna_graph* g, const std::vector<T>& v, const T** dst) {
  if (v.empty()) {
    *dst = nullptr;
    return GNA_OK;
  }
  void* p = nullptr;
  GNA_CUDA_TRY(cudaMalloc(&p, v.size() * sizeof(T)));
  g->allocations.push_back(p);
  GNA_CUDA_TRY(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *dst = (const T*)p;
  return GNA_OK;
}

}  // namespace

}  // namespace gna

namespace gna {
namespace {

// Shared by both creation entries: Jxy is the off-diagonal coupling (J of Heisenberg
// bonds), Jz / hz / cb the diagonal terms (NULL hz, cb = zero).
gna_status create_graph(int32_t n_sites, int32_t n_edges, const int32_t* edges, const double* Jz,
                        const double* Jxy, const double* hz, const double* cb, int32_t max_layers,
                        gna_graph** out) {
  if (!out) return GNA_ERR_INVALID_ARG;
  *out = nullptr;
  gna_status st = validate(n_sites, n_edges, edges, Jxy, max_layers, true);
  if (st != GNA_OK) return st;
  for (const double* a : {Jz, hz, cb}) {
    if (a == nullptr) continue;
    for (int e = 0; e < n_edges; ++e)
      if (!std::isfinite(a[e])) return GNA_ERR_INVALID_ARG;
  }
  if (n_edges > 0 && Jz == nullptr) return GNA_ERR_INVALID_ARG;
  HostGraph h;
  build(n_sites, n_edges, edges, Jxy, max_layers, &h);
  h.Jz.assign(n_edges, 0.0);
  h.hz.assign(n_edges, 0.0);
  h.cb.assign(n_edges, 0.0);
  for (int e = 0; e < n_edges; ++e) {
    h.Jz[e] = Jz[e];
    if (hz) h.hz[e] = hz[e];
    if (cb) h.cb[e] = cb[e];
  }
  gna_graph* g = new gna_graph();
  cudaGetDevice(&g->device);
  g->d.n = h.n;
  g->d.E = h.E;
  g->d.Lmax = h.Lmax;
#define UP(vec, field)                       \
  st = upload(g, vec, &g->d.field);          \
  if (st != GNA_OK) {                        \
    gna_graph_destroy(g);                    \
    return st;                               \
  }
  UP(h.row_ptr, row_ptr);
  UP(h.col, col);
  UP(h.col_edge, col_edge);
  UP(h.wf, wf);
  UP(h.wd, wd);
  UP(h.edges, edges);
  UP(h.J, J);
  UP(h.Jz, Jz);
  UP(h.hz, hz);
  UP(h.cb, cb);
  UP(h.ball_off, ball_off);
  UP(h.ball_size, ball_size);
  UP(h.ball_vert, ball_vert);
  UP(h.row_nbr, row_nbr);
  UP(h.nbr_pos, nbr_pos);
  UP(h.ball_span, ball_span);
  UP(h.row_pack, row_pack);
  UP(h.nbr_pos16, nbr_pos16);
  UP(h.bond_ent, bond_ent);
#undef UP
  g->pack_ok = h.pack_ok;
  g->h_row_ptr = h.row_ptr;
  g->h_col = h.col;
  g->h_edges = h.edges;
  g->h_ball_size = h.ball_size;
  g->h_ball_off = h.ball_off;
  g->h_J = h.J;
  g->max_ball = h.max_ball;
  g->max_span = h.max_span;
  for (int v = 0; v < h.n; ++v) g->max_deg = std::max(g->max_deg, h.row_ptr[v + 1] - h.row_ptr[v]);
  *out = g;
  return GNA_OK;
}

}  // namespace
}  // namespace gna

extern "C" gna_status gna_graph_create(int32_t n_sites, int32_t n_edges, const int32_t* edges,
                                       const double* J, int32_t max_layers, gna_graph** out) {
  return gna::create_graph(n_sites, n_edges, edges, J, J, nullptr, nullptr, max_layers, out);
}

extern "C" gna_status gna_graph_create_xxz(int32_t n_sites, int32_t n_edges, const int32_t* edges,
                                           const double* Jz, const double* Jxy, const double* hz,
                                           const double* c, int32_t max_layers, gna_graph** out) {
  if (n_edges > 0 && (Jz == nullptr || Jxy == nullptr || hz == nullptr || c == nullptr))
    return GNA_ERR_INVALID_ARG;
  return gna::create_graph(n_sites, n_edges, edges, Jz, Jxy, hz, c, max_layers, out);
}

extern "C" gna_status gna_graph_destroy(gna_graph* g) {
  if (!g) return GNA_ERR_INVALID_ARG;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != g->device) cudaSetDevice(g->device);
  for (void* p : g->allocations) cudaFree(p);
  if (cur != g->device) cudaSetDevice(cur);
  delete g;
  return GNA_OK;
}

extern "C" gna_status gna_graph_info(const gna_graph* g, int32_t* n_sites, int32_t* n_edges,
                                     int32_t* max_layers) {
  if (!g) return GNA_ERR_INVALID_ARG;
  if (n_sites) *n_sites = g->d.n;
  if (n_edges) *n_edges = g->d.E;
  if (max_layers) *max_layers = g->d.Lmax;
  return GNA_OK;
}

extern "C" gna_status gna_ball_sizes_host(int32_t n_sites, int32_t n_edges, const int32_t* edges,
                                          int32_t n_layers, int32_t* out) {
  using namespace gna;
  if (!out && n_edges > 0) return GNA_ERR_INVALID_ARG;
  gna_status st = validate(n_sites, n_edges, edges, nullptr, n_layers, false);
  if (st != GNA_OK) return st;
  HostGraph h;
  build(n_sites, n_edges, edges, nullptr, n_layers, &h);
  std::memcpy(out, h.ball_size.data(), h.ball_size.size() * sizeof(int32_t));
  return GNA_OK;
}
