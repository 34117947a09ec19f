// Planner of libvtm: wire tearing of a node partition into sub-circuits and
// the torn-port table (Sec. V, Steps 1-4), band ordering of every
// sub-circuit, and host assembly of the condensed local matrices K_P.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <queue>
#include <thread>

#include "vtm_internal.h"

namespace vtm {

static thread_local std::string g_detail;

void set_detail(const std::string& msg) { g_detail = msg; }

vtm_status dev_alloc(DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return VTM_OK;
  dev_free(b);
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    b.p = nullptr;
    set_detail(std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? VTM_ENOMEM : VTM_ECUDA;
  }
  b.bytes = bytes;
  return VTM_OK;
}

void dev_free(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
static vtm_status fetch(std::vector<T>& h, const T* src, size_t count) {
  h.resize(count);
  if (count == 0) return VTM_OK;
  if (is_device_ptr(src)) {
    VTM_CUDA_TRY(cudaMemcpy(h.data(), src, count * sizeof(T), cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(h.data(), src, count * sizeof(T));
  }
  return VTM_OK;
}

// Half bandwidth of one tile's local pattern under the ordering `loc`.
static int tile_bandwidth(const vtm_plan_s* P, const std::vector<int32_t>& nodes,
                          const std::vector<int32_t>& loc_of, int32_t tile) {
  int bw = 0;
  for (size_t a = 0; a < nodes.size(); ++a) {
    int32_t i = nodes[a];
    int li = loc_of[i];
    for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
      int32_t j = P->h_colidx[q];
      if (P->h_part[j] != tile) continue;
      int d = std::abs(loc_of[j] - li);
      bw = std::max(bw, d);
    }
  }
  return bw;
}

// Reverse Cuthill-McKee ordering of one tile (symmetrised pattern).
static void tile_rcm(const vtm_plan_s* P, const std::vector<int32_t>& nodes, int32_t tile,
                     std::vector<int32_t>& out, std::vector<int32_t>& mark) {
  const size_t m = nodes.size();
  // local adjacency
  std::vector<int32_t> deg(m, 0);
  std::vector<std::vector<int32_t>> adj(m);
  for (size_t a = 0; a < m; ++a) mark[nodes[a]] = (int32_t)a;
  for (size_t a = 0; a < m; ++a) {
    int32_t i = nodes[a];
    for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
      int32_t j = P->h_colidx[q];
      if (j == i || P->h_part[j] != tile) continue;
      int32_t b = mark[j];
      adj[a].push_back(b);
      adj[b].push_back((int32_t)a);
    }
  }
  for (size_t a = 0; a < m; ++a) {
    std::sort(adj[a].begin(), adj[a].end());
    adj[a].erase(std::unique(adj[a].begin(), adj[a].end()), adj[a].end());
    deg[a] = (int32_t)adj[a].size();
  }
  std::vector<char> seen(m, 0);
  std::vector<int32_t> order;
  order.reserve(m);
  while (order.size() < m) {
    // start: unvisited node of minimum degree (ties: lowest local id)
    int32_t s = -1;
    for (size_t a = 0; a < m; ++a)
      if (!seen[a] && (s < 0 || deg[a] < deg[s])) s = (int32_t)a;
    std::queue<int32_t> q;
    q.push(s);
    seen[s] = 1;
    while (!q.empty()) {
      int32_t a = q.front();
      q.pop();
      order.push_back(a);
      std::vector<int32_t> nb;
      for (int32_t b : adj[a])
        if (!seen[b]) {
          seen[b] = 1;
          nb.push_back(b);
        }
      std::stable_sort(nb.begin(), nb.end(), [&](int32_t x, int32_t y) { return deg[x] < deg[y]; });
      for (int32_t b : nb) q.push(b);
    }
  }
  out.resize(m);
  for (size_t a = 0; a < m; ++a) out[a] = nodes[order[m - 1 - a]];
}

// f(i) for i in [0, count), spread over the host's cores (interleaved, so that
// neighbouring items of uneven cost land on different threads).  f must only
// write state that no other i touches.
template <class F>
static void parallel_items(int64_t count, F&& f) {
  const unsigned hw = std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  const int64_t nt = std::min<int64_t>(hw, std::max<int64_t>(1, count / 16));
  if (nt <= 1) {
    for (int64_t i = 0; i < count; ++i) f(i);
    return;
  }
  std::vector<std::thread> pool;
  pool.reserve(nt);
  for (int64_t t = 0; t < nt; ++t)
    pool.emplace_back([&, t]() {
      for (int64_t i = t; i < count; i += nt) f(i);
    });
  for (auto& th : pool) th.join();
}

static int64_t csr_find(const vtm_plan_s* P, int32_t i, int32_t j) {
  const int32_t* b = P->h_colidx.data() + P->h_rowptr[i];
  const int32_t* e = P->h_colidx.data() + P->h_rowptr[i + 1];
  const int32_t* f = std::lower_bound(b, e, j);
  if (f != e && *f == j) return (int64_t)(f - P->h_colidx.data());
  return -1;
}

struct CutPair {
  int32_t lo, hi;
  int64_t pos_lohi, pos_hilo;
  bool wire;
};

static double val_at(const vtm_plan_s* P, int64_t pos) { return pos >= 0 ? P->h_vals[pos] : 0.0; }

// All structure that depends only on the pattern, the partition and the
// signs that decide which cut pairs carry a virtual line.
static vtm_status build_structure(vtm_plan_s* P, std::vector<CutPair>& pairs) {
  const int64_t n = P->n;
  const int32_t np = P->nparts;
  // tiles
  std::vector<int32_t> count(np + 1, 0);
  for (int64_t i = 0; i < n; ++i) count[P->h_part[i] + 1]++;
  for (int32_t t = 0; t < np; ++t) {
    if (count[t + 1] == 0) {
      set_detail("vtm_plan: part " + std::to_string(t) + " is empty");
      return VTM_EINVAL;
    }
    count[t + 1] += count[t];
  }
  P->node_off = count;
  std::vector<std::vector<int32_t>> tnodes(np);
  for (int64_t i = 0; i < n; ++i) tnodes[P->h_part[i]].push_back((int32_t)i);
  P->perm.assign(n, 0);
  P->iperm.assign(n, 0);
  P->bw.assign(np, 0);
  // per tile: natural or reverse Cuthill-McKee order, whichever has the smaller
  // half bandwidth; tiles in parallel (each touches only its own nodes'
  // entries of loc_of, mark, perm and iperm)
  std::vector<int32_t> loc_of(n, 0), mark(n, 0);
  parallel_items(np, [&](int64_t tt) {
    const int32_t t = (int32_t)tt;
    std::vector<int32_t> rcm;
    auto& nd = tnodes[t];
    for (size_t a = 0; a < nd.size(); ++a) loc_of[nd[a]] = (int32_t)a;
    int bw_nat = tile_bandwidth(P, nd, loc_of, t);
    std::vector<int32_t>* best = &nd;
    int bw_best = bw_nat;
    if (bw_nat > 1 && nd.size() > 2) {
      tile_rcm(P, nd, t, rcm, mark);
      for (size_t a = 0; a < rcm.size(); ++a) loc_of[rcm[a]] = (int32_t)a;
      int bw_rcm = tile_bandwidth(P, rcm, loc_of, t);
      if (bw_rcm < bw_nat) {
        best = &rcm;
        bw_best = bw_rcm;
      }
    }
    for (size_t a = 0; a < best->size(); ++a) {
      int32_t node = (*best)[a];
      P->perm[P->node_off[t] + a] = node;
      P->iperm[node] = P->node_off[t] + (int32_t)a;
    }
    P->bw[t] = bw_best;
  });
  P->max_nodes = 0;
  P->max_bw = 0;
  for (int32_t t = 0; t < np; ++t) {
    P->max_nodes = std::max<int32_t>(P->max_nodes, P->node_off[t + 1] - P->node_off[t]);
    P->max_bw = std::max(P->max_bw, P->bw[t]);
  }
  P->band_off.assign(np, 0);
  int64_t off = 0;
  for (int32_t t = 0; t < np; ++t) {
    P->band_off[t] = off;
    off += (int64_t)(P->node_off[t + 1] - P->node_off[t]) * (P->bw[t] + 1);
  }
  P->band_elems = off;

  // cut pairs (Sec. V Step 1: every branch between two parts is torn)
  pairs.clear();
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
      int32_t j = P->h_colidx[q];
      if (P->h_part[j] == P->h_part[i]) continue;
      if (i < j) {
        pairs.push_back({(int32_t)i, j, q, csr_find(P, j, (int32_t)i), false});
      } else if (csr_find(P, j, (int32_t)i) < 0) {
        pairs.push_back({j, (int32_t)i, -1, q, false});
      }
    }
  }
  std::vector<int32_t> pn, pr, pt;
  std::vector<int64_t> pij, pji;
  P->lag_i.clear();
  P->lag_j.clear();
  P->lag_pos.clear();
  for (auto& cp : pairs) {
    double a1 = val_at(P, cp.pos_lohi), a2 = val_at(P, cp.pos_hilo);
    double g = -(a1 + a2) / 2.0;
    cp.wire = P->method == VTM_METHOD_VTM && g > 0;
    double r1 = cp.wire ? a1 + g : a1;
    double r2 = cp.wire ? a2 + g : a2;
    if (r1 != 0.0) {
      P->lag_i.push_back(cp.lo);
      P->lag_j.push_back(cp.hi);
      P->lag_pos.push_back(cp.pos_lohi);
    }
    if (r2 != 0.0) {
      P->lag_i.push_back(cp.hi);
      P->lag_j.push_back(cp.lo);
      P->lag_pos.push_back(cp.pos_hilo);
    }
    if (cp.wire) {
      pn.push_back(cp.lo); pr.push_back(cp.hi); pij.push_back(cp.pos_lohi); pji.push_back(cp.pos_hilo);
      pn.push_back(cp.hi); pr.push_back(cp.lo); pij.push_back(cp.pos_hilo); pji.push_back(cp.pos_lohi);
    }
  }
  // ports: grouped by tile, then (node, remote)
  const size_t npt = pn.size();
  std::vector<int64_t> idx(npt);
  std::iota(idx.begin(), idx.end(), 0);
  std::sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) {
    int32_t ta = P->h_part[pn[a]], tb = P->h_part[pn[b]];
    if (ta != tb) return ta < tb;
    if (pn[a] != pn[b]) return pn[a] < pn[b];
    return pr[a] < pr[b];
  });
  P->port_node.resize(npt);
  P->port_remote.resize(npt);
  P->port_pos_ij.resize(npt);
  P->port_pos_ji.resize(npt);
  P->port_loc.resize(npt);
  P->port_off.assign(np + 1, 0);
  for (size_t s = 0; s < npt; ++s) {
    int64_t a = idx[s];
    P->port_node[s] = pn[a];
    P->port_remote[s] = pr[a];
    P->port_pos_ij[s] = pij[a];
    P->port_pos_ji[s] = pji[a];
    int32_t t = P->h_part[pn[a]];
    P->port_loc[s] = P->iperm[pn[a]] - P->node_off[t];
    P->port_off[t + 1]++;
  }
  for (int32_t t = 0; t < np; ++t) P->port_off[t + 1] += P->port_off[t];
  // twins: the port whose (node, remote) is our (remote, node)
  std::vector<int64_t> key(npt), srt(npt);
  for (size_t s = 0; s < npt; ++s) key[s] = (int64_t)P->port_node[s] * n + P->port_remote[s];
  std::iota(srt.begin(), srt.end(), 0);
  std::sort(srt.begin(), srt.end(), [&](int64_t a, int64_t b) { return key[a] < key[b]; });
  P->port_twin.resize(npt);
  for (size_t s = 0; s < npt; ++s) {
    int64_t want = (int64_t)P->port_remote[s] * n + P->port_node[s];
    auto it = std::lower_bound(srt.begin(), srt.end(), want,
                               [&](int64_t a, int64_t v) { return key[a] < v; });
    if (it == srt.end() || key[*it] != want) {
      set_detail("vtm_plan: internal: twin port not found");
      return VTM_EINTERNAL;
    }
    P->port_twin[s] = (int32_t)*it;
  }
  // node runs (ports of one node are adjacent)
  P->port_run.assign(npt, 0);
  for (size_t s = 0; s < npt;) {
    size_t e = s + 1;
    int32_t t = P->h_part[P->port_node[s]];
    while (e < npt && P->port_node[e] == P->port_node[s] && (int64_t)e < P->port_off[t + 1]) ++e;
    P->port_run[s] = (uint8_t)std::min<size_t>(e - s, 255);
    if (e - s > 255) {
      set_detail("vtm_plan: more than 255 torn branches at one node");
      return VTM_EINVAL;
    }
    s = e;
  }
  // reflection-matrix layout: T^T blocks with rows padded to 8 elements
  P->T_ld.assign(np, 0);
  P->T_off.assign(np, 0);
  P->Tp_off.assign(np, 0);
  int64_t toff = 0, tpoff = 0;
  P->sum_p2 = 0;
  P->sum_tri = 0;
  P->max_ports = 0;
  for (int32_t t = 0; t < np; ++t) {
    int32_t p = P->port_off[t + 1] - P->port_off[t];
    int32_t ld = (p + 7) / 8 * 8;
    P->T_ld[t] = ld;
    P->T_off[t] = toff;
    toff += (int64_t)p * ld;
    P->sum_p2 += (int64_t)p * p;
    P->sum_tri += (int64_t)p * (p + 1) / 2;
    P->max_ports = std::max(P->max_ports, p);
    const int64_t nb = (p + kSymB - 1) / kSymB;
    P->Tp_off[t] = tpoff;
    tpoff += nb * (nb + 1) / 2 * kSymB * kSymB;
  }
  P->T_elems = toff;
  P->Tp_elems = tpoff;
  return VTM_OK;
}

// True if the current values give the same torn lines and the same set of
// lagged positions as the ones the plan was built with.
static bool same_cut_structure(const vtm_plan_s* P) {
  std::vector<int64_t> wires, lags;
  for (int64_t i = 0; i < P->n; ++i) {
    for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
      int32_t j = P->h_colidx[q];
      if (P->h_part[j] == P->h_part[i]) continue;
      int64_t back = csr_find(P, j, (int32_t)i);
      if (i > j && back >= 0) continue;
      int64_t p1 = i < j ? q : back, p2 = i < j ? back : q;
      double a1 = val_at(P, p1), a2 = val_at(P, p2);
      double g = -(a1 + a2) / 2.0;
      bool wire = P->method == VTM_METHOD_VTM && g > 0;
      if (wire) wires.push_back(p1 >= 0 ? p1 : p2);
      double r1 = wire ? a1 + g : a1, r2 = wire ? a2 + g : a2;
      if (r1 != 0.0) lags.push_back(p1);
      if (r2 != 0.0) lags.push_back(p2);
    }
  }
  std::vector<int64_t> w0, l0;
  for (size_t s = 0; s < P->port_node.size(); ++s)
    if (P->port_node[s] < P->port_remote[s])
      w0.push_back(P->port_pos_ij[s] >= 0 ? P->port_pos_ij[s] : P->port_pos_ji[s]);
  for (size_t q = 0; q < P->lag_pos.size(); ++q) l0.push_back(P->lag_pos[q]);
  std::sort(wires.begin(), wires.end());
  std::sort(lags.begin(), lags.end());
  std::sort(w0.begin(), w0.end());
  std::sort(l0.begin(), l0.end());
  // a lagged entry may vanish (rho = 0) but no new one may appear
  if (wires != w0) return false;
  return std::includes(l0.begin(), l0.end(), lags.begin(), lags.end());
}

// Diagonal of the partial input admittance S~ = C - E~ D~^-1 F~ of every port
// (Sec. VIII, choice 5): D~ is D_P = A_PP + sum_s g_s e_l e_l^T restricted to
// the nodes of the sub-circuit within `radius` branches of the port's node;
// S~_ss = 2 g_s - 4 g_s^2 [D~^-1]_(l,l), by a dense LU with partial pivoting.
static vtm_status schur_diag_ports(vtm_plan_s* P, int radius, std::vector<double>& S) {
  const size_t npt = P->port_node.size();
  S.assign(npt, 0.0);
  std::vector<double> gsum(P->n, 0.0);
  for (size_t s = 0; s < npt; ++s) gsum[P->port_node[s]] += P->port_g[s];
  std::vector<int32_t> mark(P->n, -1), sel;
  std::vector<double> D, z;
  for (size_t s = 0; s < npt; ++s) {
    const int32_t l = P->port_node[s], t = P->h_part[l];
    sel.assign(1, l);
    mark[l] = (int32_t)s;
    size_t lo = 0;
    for (int r = 0; r < radius; ++r) {
      const size_t hi = sel.size();
      for (size_t q = lo; q < hi; ++q) {
        const int32_t i = sel[q];
        for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) {
          const int32_t j = P->h_colidx[e];
          if (P->h_part[j] == t && mark[j] != (int32_t)s) {
            mark[j] = (int32_t)s;
            sel.push_back(j);
          }
        }
      }
      lo = hi;
    }
    const int m = (int)sel.size();
    if (m > 512) {
      set_detail("vtm_set_admittance: the neighbourhood of a port exceeds 512 nodes; lower radius");
      return VTM_EINVAL;
    }
    std::vector<int32_t> pos(m);
    D.assign((size_t)m * m, 0.0);
    for (int a = 0; a < m; ++a) {
      const int32_t i = sel[a];
      for (int64_t e = P->h_rowptr[i]; e < P->h_rowptr[i + 1]; ++e) {
        const int32_t j = P->h_colidx[e];
        if (P->h_part[j] != t || mark[j] != (int32_t)s) continue;
        const int b = (int)(std::find(sel.begin(), sel.end(), j) - sel.begin());
        D[(size_t)a * m + b] += P->h_vals[e];
      }
      D[(size_t)a * m + a] += gsum[i];
    }
    // solve D z = e_0 (the port's node is sel[0])
    z.assign(m, 0.0);
    z[0] = 1.0;
    for (int c = 0; c < m; ++c) {
      int piv = c;
      for (int r = c + 1; r < m; ++r)
        if (std::fabs(D[(size_t)r * m + c]) > std::fabs(D[(size_t)piv * m + c])) piv = r;
      if (D[(size_t)piv * m + c] == 0.0) {
        set_detail("vtm_set_admittance: singular partial sub-circuit matrix");
        return VTM_ESINGULAR;
      }
      if (piv != c) {
        for (int k = 0; k < m; ++k) std::swap(D[(size_t)c * m + k], D[(size_t)piv * m + k]);
        std::swap(z[c], z[piv]);
      }
      for (int r = c + 1; r < m; ++r) {
        const double f = D[(size_t)r * m + c] / D[(size_t)c * m + c];
        if (f == 0.0) continue;
        for (int k = c; k < m; ++k) D[(size_t)r * m + k] -= f * D[(size_t)c * m + k];
        z[r] -= f * z[c];
      }
    }
    for (int c = m - 1; c >= 0; --c) {
      double acc = z[c];
      for (int k = c + 1; k < m; ++k) acc -= D[(size_t)c * m + k] * z[k];
      z[c] = acc / D[(size_t)c * m + c];
    }
    const double g = P->port_g[s];
    S[s] = 2 * g - 4 * g * g * z[0];
  }
  return VTM_OK;
}

// Admittance of every line from the plan's choice (Sec. VIII); both ports of
// a line get the same value.
static vtm_status line_admittance(vtm_plan_s* P) {
  const size_t npt = P->port_node.size();
  P->port_W.assign(npt, P->W);
  switch (P->w_kind) {
    case VTM_W_ALPHA:
      break;
    case VTM_W_DIAG:
      for (size_t s = 0; s < npt; ++s) P->port_W[s] = 2.0 * P->port_g[s];
      break;
    case VTM_W_WOB:
      for (size_t s = 0; s < npt; ++s) P->port_W[s] = P->w_alpha * 2.0 * P->port_g[s];
      break;
    case VTM_W_SCA: {
      std::vector<double> S;
      VTM_TRY(schur_diag_ports(P, P->w_radius, S));
      for (size_t s = 0; s < npt; ++s) {
        const int32_t tw = P->port_twin[s];
        const bool low = P->h_part[P->port_node[s]] <= P->h_part[P->port_node[tw]];
        P->port_W[s] = low ? S[s] : S[tw];
      }
      break;
    }
    case VTM_W_LINE:
      P->port_W = P->w_user;
      break;
    default:
      return VTM_EINVAL;
  }
  for (size_t s = 0; s < npt; ++s)
    if (!(P->port_W[s] > 0) || !std::isfinite(P->port_W[s])) {
      set_detail("line admittance not positive at port " + std::to_string(s));
      return VTM_EINVAL;
    }
  return VTM_OK;
}

// Values: branch conductances, line admittances, the per-port coefficients,
// lagged couplings and the band of K_P.
vtm_status assemble_local(vtm_plan_s* P) {
  const int32_t np = P->nparts;
  const size_t npt = P->port_node.size();
  P->port_g.resize(npt);
  for (size_t s = 0; s < npt; ++s) {
    double g = -(val_at(P, P->port_pos_ij[s]) + val_at(P, P->port_pos_ji[s])) / 2.0;
    if (!(g > 0)) {
      set_detail("vtm_set_values: a torn branch lost its positive conductance");
      return VTM_EINVAL;
    }
    P->port_g[s] = g;
  }
  if (P->w_dirty || P->port_W.size() != npt) {
    VTM_TRY(line_admittance(P));
    P->w_dirty = false;
  }
  // waves are carried as w / d_s with d_s = sqrt(W_s / W_ref): for one W on
  // every line d = 1; otherwise d = sqrt(W_s) (power waves), which keeps the
  // condensed operator symmetric for a symmetric A
  const bool scalar_w = P->w_kind == VTM_W_ALPHA;
  std::vector<double> beta(npt), bin(npt), bout(npt), rho(npt), kd(2 * npt);
  std::vector<float> kd32(2 * npt);
  std::vector<float> kddf(4 * npt);  // (g/W, d) as double-float pairs (kernel 12)
  P->port_d.assign(npt, 1.0);
  for (size_t s = 0; s < npt; ++s) {
    const double g = P->port_g[s], W = P->port_W[s];
    const double d = scalar_w ? 1.0 : std::sqrt(W);
    P->port_d[s] = d;
    beta[s] = 2 * g / (2 * g + W);
    bin[s] = scalar_w ? beta[s] : beta[s] * d;
    bout[s] = scalar_w ? 2.0 * W * beta[s] : 2.0 * W * beta[s] / d;
    rho[s] = (W - 2.0 * g) / (W + 2.0 * g);
    kd[2 * s] = g / W;
    kd[2 * s + 1] = d;
    kd32[2 * s] = (float)(g / W);
    kd32[2 * s + 1] = (float)d;
    kddf[4 * s] = (float)(g / W);
    kddf[4 * s + 1] = (float)(g / W - (double)kddf[4 * s]);
    kddf[4 * s + 2] = (float)d;
    kddf[4 * s + 3] = (float)(d - (double)kddf[4 * s + 2]);
  }
  P->lag_rho.resize(P->lag_i.size());
  for (size_t q = 0; q < P->lag_i.size(); ++q) {
    // remainder after the branch part (if the pair carries a line)
    int32_t i = P->lag_i[q], j = P->lag_j[q];
    int64_t pji = csr_find(P, j, i);
    double a = val_at(P, P->lag_pos[q]);
    double g = -(a + val_at(P, pji)) / 2.0;
    P->lag_rho[q] = (P->method == VTM_METHOD_VTM && g > 0) ? a + g : a;
  }
  std::vector<double> Lc(P->band_elems, 0.0), Uc;
  if (!P->symmetric) Uc.assign(P->band_elems, 0.0);
  for (int32_t t = 0; t < np; ++t) {
    const int32_t B = P->bw[t] + 1;
    const int32_t off = P->node_off[t];
    const int32_t cnt = P->node_off[t + 1] - off;
    double* lc = Lc.data() + P->band_off[t];
    double* uc = P->symmetric ? nullptr : Uc.data() + P->band_off[t];
    for (int32_t l = 0; l < cnt; ++l) {
      int32_t i = P->perm[off + l];
      for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
        int32_t j = P->h_colidx[q];
        if (P->h_part[j] != t) continue;
        int32_t m = P->iperm[j] - off;
        if (m <= l) {
          lc[(int64_t)m * B + (l - m)] += P->h_vals[q];
        } else if (uc) {
          uc[(int64_t)m * B + (m - l)] += P->h_vals[q];
        }
      }
    }
    for (int32_t s = P->port_off[t]; s < P->port_off[t + 1]; ++s) {
      const double g = P->port_g[s], W = P->port_W[s];
      lc[(int64_t)P->port_loc[s] * B] += g - 4 * g * g / (2 * g + W);
    }
  }
  cudaStream_t st = P->stream;
  VTM_TRY(upload(P->d_Lc, Lc, st));
  if (!P->symmetric) {
    VTM_TRY(upload(P->d_Uc, Uc, st));
  } else {
    VTM_TRY(dev_alloc(P->d_Uc, std::max<size_t>(16, Lc.size() * sizeof(double))));
  }
  VTM_TRY(upload(P->d_beta, bin, st));
  VTM_TRY(upload(P->d_bout, bout, st));
  // FP32 copies for the port-wise kernels of the low-precision batched path
  {
    std::vector<float> b32(bin.begin(), bin.end()), o32(bout.begin(), bout.end());
    VTM_TRY(upload(P->d_beta32, b32, st));
    VTM_TRY(upload(P->d_bout32, o32, st));
    VTM_CUDA_TRY(cudaStreamSynchronize(st));  // the host vectors are about to go
  }
  VTM_TRY(upload(P->d_rho, rho, st));
  VTM_TRY(upload(P->d_kd, kd, st));
  VTM_TRY(upload(P->d_kd32, kd32, st));
  VTM_TRY(upload(P->d_kddf, kddf, st));
  if (P->general) {
    // per input: residual coefficients (g/W and d of a port, rho of a lagged
    // entry) and right-hand-side weight (beta d or -rho); per output: scale
    // (2 W beta / d or 1) and the diagonal reflection term of a port
    std::vector<double> coef(P->n_in), dsc(P->n_in, 0.0), sigma(P->n_in), scale(P->n_out),
        diag(P->n_out, 0.0);
    for (int64_t a = 0; a < P->n_in; ++a) {
      const int32_t it = P->in_item[a];
      if (P->in_kind[a] == 0) {
        coef[a] = kd[2 * it];
        dsc[a] = kd[2 * it + 1];
        sigma[a] = bin[it];
      } else {
        coef[a] = P->lag_rho[it];
        sigma[a] = -P->lag_rho[it];
      }
    }
    for (int64_t o = 0; o < P->n_out; ++o) {
      const int32_t it = P->out_item[o];
      if (it >= 0) {
        scale[o] = bout[it];
        diag[o] = rho[it];
      } else {
        scale[o] = 1.0;
      }
    }
    VTM_TRY(upload(P->d_in_coef, coef, st));
    VTM_TRY(upload(P->d_in_d, dsc, st));
    VTM_TRY(upload(P->d_in_sigma, sigma, st));
    VTM_TRY(upload(P->d_out_scale, scale, st));
    VTM_TRY(upload(P->d_out_diag, diag, st));
  }
  VTM_CUDA_TRY(cudaStreamSynchronize(st));
  return VTM_OK;
}

// Channel tables of the general form (see vtm_internal.h).
static vtm_status build_general(vtm_plan_s* P) {
  const int32_t np = P->nparts;
  const int64_t nl = (int64_t)P->lag_i.size();
  // lagged entries grouped by the tile of their row, ordered by (row, column)
  std::vector<int64_t> lag_order(nl);
  std::iota(lag_order.begin(), lag_order.end(), 0);
  std::sort(lag_order.begin(), lag_order.end(), [&](int64_t a, int64_t b) {
    int32_t ta = P->h_part[P->lag_i[a]], tb = P->h_part[P->lag_i[b]];
    if (ta != tb) return ta < tb;
    if (P->lag_i[a] != P->lag_i[b]) return P->lag_i[a] < P->lag_i[b];
    return P->lag_j[a] < P->lag_j[b];
  });
  // probes: distinct columns of lagged entries, grouped by their tile
  std::vector<int32_t> probe_nodes;
  for (int64_t q = 0; q < nl; ++q) probe_nodes.push_back(P->lag_j[q]);
  std::sort(probe_nodes.begin(), probe_nodes.end(), [&](int32_t a, int32_t b) {
    int32_t ta = P->h_part[a], tb = P->h_part[b];
    return ta != tb ? ta < tb : a < b;
  });
  probe_nodes.erase(std::unique(probe_nodes.begin(), probe_nodes.end()), probe_nodes.end());
  std::vector<int32_t> nlag(np, 0), nprobe(np, 0);
  for (int64_t q = 0; q < nl; ++q) nlag[P->h_part[P->lag_i[q]]]++;
  for (int32_t v : probe_nodes) nprobe[P->h_part[v]]++;
  P->in_off.assign(np + 1, 0);
  P->out_off.assign(np + 1, 0);
  for (int32_t t = 0; t < np; ++t) {
    const int32_t p = P->port_off[t + 1] - P->port_off[t];
    P->in_off[t + 1] = P->in_off[t] + p + nlag[t];
    P->out_off[t + 1] = P->out_off[t] + p + nprobe[t];
  }
  P->n_in = P->in_off[np];
  P->n_out = P->out_off[np];
  // output slot of each probe node
  std::vector<int32_t> probe_slot(P->n, -1);
  {
    std::vector<int32_t> fill(np, 0);
    for (int32_t v : probe_nodes) {
      const int32_t t = P->h_part[v];
      const int32_t p = P->port_off[t + 1] - P->port_off[t];
      probe_slot[v] = P->out_off[t] + p + fill[t]++;
    }
  }
  P->in_src.assign(P->n_in, -1);
  P->in_kind.assign(P->n_in, 0);
  P->in_twin.assign(P->n_in, -1);
  P->in_own_out.assign(P->n_in, -1);
  P->in_loc.assign(P->n_in, 0);
  P->in_item.assign(P->n_in, -1);
  P->out_loc.assign(P->n_out, 0);
  P->out_item.assign(P->n_out, -1);
  // global input / output id of a port
  auto port_in = [&](int32_t s) {
    const int32_t t = P->h_part[P->port_node[s]];
    return P->in_off[t] + (s - P->port_off[t]);
  };
  auto port_out = [&](int32_t s) {
    const int32_t t = P->h_part[P->port_node[s]];
    return P->out_off[t] + (s - P->port_off[t]);
  };
  for (int32_t s = 0; s < (int32_t)P->port_node.size(); ++s) {
    const int32_t a = port_in(s), o = port_out(s);
    const int32_t tw = P->port_twin[s];
    P->in_kind[a] = 0;
    P->in_src[a] = port_out(tw);
    P->in_twin[a] = port_in(tw);
    P->in_own_out[a] = o;
    P->in_loc[a] = P->port_loc[s];
    P->in_item[a] = s;
    P->out_loc[o] = P->port_loc[s];
    P->out_item[o] = s;
  }
  {
    std::vector<int32_t> fill(np, 0);
    for (int64_t k = 0; k < nl; ++k) {
      const int64_t q = lag_order[k];
      const int32_t i = P->lag_i[q], j = P->lag_j[q];
      const int32_t t = P->h_part[i];
      const int32_t p = P->port_off[t + 1] - P->port_off[t];
      const int32_t a = P->in_off[t] + p + fill[t]++;
      P->in_kind[a] = 1;
      P->in_src[a] = probe_slot[j];
      P->in_loc[a] = P->iperm[i] - P->node_off[t];
      P->in_item[a] = (int32_t)q;
    }
  }
  for (int32_t v : probe_nodes) {
    const int32_t o = probe_slot[v];
    const int32_t t = P->h_part[v];
    P->out_loc[o] = P->iperm[v] - P->node_off[t];
    P->out_item[o] = -1;
  }
  // residual runs: inputs of each tile sorted by their row node
  P->res_perm.assign(P->n_in, 0);
  P->res_run.assign(P->n_in, 0);
  P->max_in = P->max_out = 0;
  for (int32_t t = 0; t < np; ++t) {
    const int32_t a0 = P->in_off[t], ni = P->in_off[t + 1] - a0;
    P->max_in = std::max(P->max_in, ni);
    P->max_out = std::max(P->max_out, P->out_off[t + 1] - P->out_off[t]);
    std::vector<int32_t> idx(ni);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(),
                     [&](int32_t x, int32_t y) { return P->in_loc[a0 + x] < P->in_loc[a0 + y]; });
    for (int32_t k = 0; k < ni;) {
      int32_t e = k + 1;
      while (e < ni && P->in_loc[a0 + idx[e]] == P->in_loc[a0 + idx[k]]) ++e;
      if (e - k > 255) {
        set_detail("vtm_plan: more than 255 cut couplings in one row");
        return VTM_EINVAL;
      }
      P->res_run[a0 + k] = (uint8_t)(e - k);
      k = e;
    }
    for (int32_t k = 0; k < ni; ++k) P->res_perm[a0 + k] = idx[k];
  }
  // operator layout: per tile, one row of E^T per input, rows padded to 8
  P->E_ld.assign(np, 0);
  P->E_off.assign(np, 0);
  int64_t off = 0;
  for (int32_t t = 0; t < np; ++t) {
    const int32_t ni = P->in_off[t + 1] - P->in_off[t];
    const int32_t no = P->out_off[t + 1] - P->out_off[t];
    P->E_ld[t] = (no + 7) / 8 * 8;
    P->E_off[t] = off;
    off += (int64_t)ni * P->E_ld[t];
  }
  P->E_elems = off;
  cudaStream_t st = P->stream;
  std::vector<int32_t> in_tile(P->n_in);
  for (int32_t t = 0; t < np; ++t)
    for (int32_t a = P->in_off[t]; a < P->in_off[t + 1]; ++a) in_tile[a] = t;
  VTM_TRY(upload(P->d_in_off, P->in_off, st));
  VTM_TRY(upload(P->d_out_off, P->out_off, st));
  VTM_TRY(upload(P->d_in_src, P->in_src, st));
  VTM_TRY(upload(P->d_in_kind, P->in_kind, st));
  VTM_TRY(upload(P->d_in_twin, P->in_twin, st));
  VTM_TRY(upload(P->d_in_own_out, P->in_own_out, st));
  VTM_TRY(upload(P->d_in_loc, P->in_loc, st));
  VTM_TRY(upload(P->d_res_perm, P->res_perm, st));
  VTM_TRY(upload(P->d_res_run, P->res_run, st));
  VTM_TRY(upload(P->d_out_loc, P->out_loc, st));
  VTM_TRY(upload(P->d_E_off, P->E_off, st));
  VTM_TRY(upload(P->d_E_ld, P->E_ld, st));
  VTM_TRY(upload(P->d_in_tile, in_tile, st));
  VTM_TRY(dev_alloc(P->d_cg, std::max<int64_t>(P->n_out, 1) * sizeof(double)));
  VTM_TRY(dev_alloc(P->d_gin, 2 * std::max<int64_t>(P->n_in, 1) * sizeof(double)));
  VTM_TRY(dev_alloc(P->d_gout, 2 * std::max<int64_t>(P->n_out, 1) * sizeof(double)));
  VTM_CUDA_TRY(cudaStreamSynchronize(st));
  return VTM_OK;
}

}  // namespace vtm

using namespace vtm;

std::vector<DevBuf*> vtm_plan_s::all_bufs() {
  return {&tabs.node_off, &tabs.bw, &tabs.band_off, &tabs.port_off, &tabs.T_off, &tabs.T_ld,
          &tabs.order, &d_rowptr, &d_colidx, &d_vals, &d_perm, &d_iperm, &d_Lc, &d_Uc, &d_Lc32, &d_Uc32, &d_v32, &d_v32b, &d_ell_val, &d_ell_col, &d_ell_len,
          &d_port_loc, &d_port_pos, &d_tdesc,
          &d_twin, &d_beta, &d_bout, &d_beta32, &d_bout32, &d_rho, &d_kd, &d_kd32, &d_run, &d_T64, &d_T32, &d_T16, &d_Tp32, &d_Tp16, &d_Tpdf, &d_dfstate, &d_cdf, &d_kddf, &d_nbr_off, &d_nbr, &d_done, &d_flow, &d_part4, &d_fstate32, &d_c64, &d_c32, &d_state64,
          &d_state32, &d_v, &d_v2, &d_xacc, &d_r, &d_bcol, &d_partials, &d_ctrl, &d_hist,
          &d_err, &d_red, &d_in_off, &d_out_off, &d_in_src, &d_in_kind, &d_in_twin,
          &d_in_own_out, &d_in_loc, &d_res_perm, &d_res_run, &d_out_loc, &d_in_coef, &d_in_d,
          &d_in_sigma, &d_out_scale, &d_out_diag, &d_E_off, &d_E_ld, &d_E, &d_cg, &d_gin,
          &d_gout, &d_in_tile, &d_item_tile, &d_item_m0, &d_item_order, &d_tc_items, &d_tc_off, &d_tc_order, &d_Ttc, &d_bk_W, &d_bk_goff, &d_bk_order, &d_bk_blk, &d_bk_Gf, &d_bk_Gb, &d_vals_df, &d_bdf, &d_xdf, &d_bexp, &d_bres2, &d_bV, &d_bV32, &d_bV32b, &d_bstate,
          &d_bc, &d_bpart,
          &d_btol2, &d_bctrl, &d_bres, &d_stage_in[0], &d_stage_in[1], &d_stage_in[2],
          &d_stage_out[0], &d_stage_out[1], &d_stage_out[2]};
}

static void fill_default_opts(vtm_opts* o) {
  if (o->max_sweeps <= 0) o->max_sweeps = 200000;
  if (o->check_every <= 0) o->check_every = 32;
  if (o->max_outer <= 0) o->max_outer = 40;
  if (o->precision < 0 || o->precision > 3) o->precision = 0;
  if (o->wait_polls <= 0) o->wait_polls = 1 << 22;
}

extern "C" vtm_status vtm_set_admittance(vtm_plan_t P, int kind, double alpha, int radius,
                                         const double* W) {
  if (!P) return VTM_EINVAL;
  const size_t npt = P->port_node.size();
  std::vector<double> user;
  switch (kind) {
    case VTM_W_ALPHA:
    case VTM_W_WOB:
      if (!(alpha > 0) || !std::isfinite(alpha)) {
        set_detail("vtm_set_admittance: alpha must be positive");
        return VTM_EINVAL;
      }
      break;
    case VTM_W_DIAG:
      break;
    case VTM_W_SCA:
      if (radius < 0 || radius > 8) {
        set_detail("vtm_set_admittance: radius must be 0..8");
        return VTM_EINVAL;
      }
      break;
    case VTM_W_LINE: {
      if (!W && npt > 0) {
        set_detail("vtm_set_admittance: VTM_W_LINE needs W[nports]");
        return VTM_EINVAL;
      }
      VTM_TRY(fetch(user, W, npt));
      for (size_t s = 0; s < npt; ++s)
        if (!(user[s] > 0) || !std::isfinite(user[s]) || user[s] != user[P->port_twin[s]]) {
          set_detail("vtm_set_admittance: W must be positive and equal at both ports of a line "
                     "(port " + std::to_string(s) + ")");
          return VTM_EINVAL;
        }
      break;
    }
    default:
      set_detail("vtm_set_admittance: unknown kind");
      return VTM_EINVAL;
  }
  const int o_kind = P->w_kind, o_radius = P->w_radius;
  const double o_alpha = P->w_alpha, o_W = P->W;
  std::vector<double> o_user = P->w_user;
  P->w_kind = kind;
  P->w_alpha = alpha;
  P->w_radius = radius;
  P->w_user = std::move(user);
  if (kind == VTM_W_ALPHA) P->W = alpha;
  P->w_dirty = true;
  vtm_status st = assemble_local(P);
  if (st != VTM_OK) {
    P->w_kind = o_kind;
    P->w_alpha = o_alpha;
    P->w_radius = o_radius;
    P->w_user = std::move(o_user);
    P->W = o_W;
    P->w_dirty = true;
    assemble_local(P);
    return st;
  }
  P->factored = false;
  if (P->transposed) {
    vtm_destroy(P->transposed);
    P->transposed = nullptr;
  }
  return VTM_OK;
}

extern "C" vtm_status vtm_get_admittance(vtm_plan_t P, double* W) {
  if (!P || !W) return VTM_EINVAL;
  const size_t npt = P->port_node.size();
  if (npt == 0) return VTM_OK;
  if (is_device_ptr(W)) {
    VTM_CUDA_TRY(cudaMemcpy(W, P->port_W.data(), npt * sizeof(double), cudaMemcpyHostToDevice));
  } else {
    std::copy(P->port_W.begin(), P->port_W.end(), W);
  }
  return VTM_OK;
}

extern "C" vtm_status vtm_set_opts(vtm_plan_t P, const vtm_opts* opts) {
  if (!P) return VTM_EINVAL;
  vtm_opts o{};
  if (opts) o = *opts;
  if (o.precision < 0 || o.precision > 3 || o.history_len < 0 || (o.history_len > 0 && !o.history)) {
    set_detail("vtm_set_opts: bad precision or history");
    return VTM_EINVAL;
  }
  if (o.sweep_kernel < 0 || o.sweep_kernel > 12) {
    set_detail("vtm_set_opts: sweep_kernel must be 0..12");
    return VTM_EINVAL;
  }
  if (o.method < 0 || o.method > 2 || ((o.method == VTM_METHOD_BJ) != (P->method == VTM_METHOD_BJ))) {
    set_detail("vtm_set_opts: method must be 0..2, and block Jacobi is chosen by vtm_plan");
    return VTM_EINVAL;
  }
  if (o.batch_solve < 0 || o.batch_solve > 3) {
    set_detail("vtm_set_opts: batch_solve must be 0, 1, 2 or 3");
    return VTM_EINVAL;
  }
  if (o.batch_kernel < 0 || o.batch_kernel > 5 || o.wait_polls < 0 || (o.flow_lag != 0 && o.flow_lag != -1) ||
      o.band_solve < 0 || o.band_solve > 1) {
    set_detail("vtm_set_opts: batch_kernel must be 0..5, wait_polls >= 0, flow_lag 0 or -1, band_solve 0 or 1");
    return VTM_EINVAL;
  }
  bool prec_changed = o.precision != P->opts.precision;
  fill_default_opts(&o);
  P->opts = o;
  if (o.history_len > P->hist_cap) {
    VTM_TRY(dev_alloc(P->d_hist, sizeof(double) * (size_t)o.history_len));
    P->hist_cap = o.history_len;
  }
  if (prec_changed && P->factored && o.precision != VTM_PREC_FP64) {
    // low-precision copies are built by vtm_factor
    P->factored = false;
  }
  return VTM_OK;
}

extern "C" vtm_status vtm_plan(int64_t n, const int64_t* rowptr, const int32_t* colidx,
                               const double* vals, const int32_t* partition, int32_t nparts,
                               double Zc, const vtm_opts* opts, void* stream, vtm_plan_t* out) {
  if (!out) return VTM_EINVAL;
  *out = nullptr;
  if (n <= 0 || n > INT32_MAX - 1 || nparts <= 0 || nparts > n || !rowptr || !colidx || !vals ||
      !partition || !(Zc > 0) || !std::isfinite(Zc)) {
    set_detail("vtm_plan: bad n, nparts, Zc or NULL array");
    return VTM_EINVAL;
  }
  vtm_plan_s* P = new (std::nothrow) vtm_plan_s();
  if (!P) return VTM_ENOMEM;
  P->n = n;
  P->nparts = nparts;
  P->Zc = Zc;
  P->W = 1.0 / Zc;
  P->stream = static_cast<cudaStream_t>(stream);
  cudaGetDevice(&P->device);
  auto fail = [&](vtm_status s) {
    vtm_destroy(P);
    return s;
  };
  vtm_status st;
  if ((st = fetch(P->h_rowptr, rowptr, (size_t)n + 1)) != VTM_OK) return fail(st);
  int64_t nnz = P->h_rowptr[n];
  if (P->h_rowptr[0] != 0 || nnz < 0) {
    set_detail("vtm_plan: rowptr[0] must be 0");
    return fail(VTM_EINVAL);
  }
  for (int64_t i = 0; i < n; ++i)
    if (P->h_rowptr[i + 1] < P->h_rowptr[i]) {
      set_detail("vtm_plan: rowptr not monotone");
      return fail(VTM_EINVAL);
    }
  P->nnz = nnz;
  if ((st = fetch(P->h_colidx, colidx, (size_t)nnz)) != VTM_OK) return fail(st);
  if ((st = fetch(P->h_vals, vals, (size_t)nnz)) != VTM_OK) return fail(st);
  if ((st = fetch(P->h_part, partition, (size_t)n)) != VTM_OK) return fail(st);
  for (int64_t i = 0; i < n; ++i) {
    if (P->h_part[i] < 0 || P->h_part[i] >= nparts) {
      set_detail("vtm_plan: partition value out of range at node " + std::to_string(i));
      return fail(VTM_EINVAL);
    }
    for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
      int32_t j = P->h_colidx[q];
      if (j < 0 || j >= n || (q > P->h_rowptr[i] && j <= P->h_colidx[q - 1])) {
        set_detail("vtm_plan: column indices out of range or not strictly increasing in row " +
                   std::to_string(i));
        return fail(VTM_EINVAL);
      }
      if (!std::isfinite(P->h_vals[q])) {
        set_detail("vtm_plan: non-finite matrix value");
        return fail(VTM_EINVAL);
      }
    }
  }
  // symmetric values -> Cholesky, else LU without pivoting (row blocks in parallel)
  {
    const int64_t nblk = (n + 4095) / 4096;
    std::vector<char> asym(nblk, 0);
    parallel_items(nblk, [&](int64_t blk) {
      for (int64_t i = blk * 4096; i < std::min<int64_t>(n, (blk + 1) * 4096) && !asym[blk]; ++i)
        for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
          int32_t j = P->h_colidx[q];
          if (j <= i) continue;
          int64_t t = csr_find(P, j, (int32_t)i);
          if (t < 0 || P->h_vals[t] != P->h_vals[q]) {
            asym[blk] = 1;
            break;
          }
        }
    });
    P->symmetric = std::find(asym.begin(), asym.end(), (char)1) == asym.end();
  }
  vtm_opts o{};
  if (opts) o = *opts;
  if (o.method != VTM_METHOD_VTM && o.method != VTM_METHOD_BJ && o.method != VTM_METHOD_ASYNC) {
    set_detail("vtm_plan: unknown method");
    return fail(VTM_EINVAL);
  }
  // asynchronous VTM tears like VTM; only its sweeps differ
  P->method = o.method == VTM_METHOD_BJ ? VTM_METHOD_BJ : VTM_METHOD_VTM;
  std::vector<CutPair> pairs;
  if ((st = build_structure(P, pairs)) != VTM_OK) return fail(st);
  P->general = !P->lag_i.empty() || P->method == VTM_METHOD_BJ;
  if (P->general && (st = build_general(P)) != VTM_OK) return fail(st);

  P->opts.precision = o.precision;
  if ((st = vtm_set_opts(P, &o)) != VTM_OK) return fail(st);

  cudaStream_t s = P->stream;
  // device tables
  if ((st = upload(P->d_rowptr, P->h_rowptr, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->d_colidx, P->h_colidx, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->d_vals, P->h_vals, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->d_perm, P->perm, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->tabs.node_off, P->node_off, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->tabs.bw, P->bw, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->tabs.band_off, P->band_off, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->tabs.port_off, P->port_off, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->tabs.T_off, P->T_off, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->tabs.T_ld, P->T_ld, s)) != VTM_OK) return fail(st);
  std::vector<int32_t> order(nparts);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return (P->port_off[a + 1] - P->port_off[a]) > (P->port_off[b + 1] - P->port_off[b]);
  });
  if ((st = upload(P->tabs.order, order, s)) != VTM_OK) return fail(st);
  std::vector<TileDesc> tdesc(nparts);
  for (int32_t i = 0; i < nparts; ++i) {
    const int32_t t = order[i];
    tdesc[i] = TileDesc{t, P->port_off[t], P->port_off[t + 1] - P->port_off[t], P->T_ld[t],
                        P->T_off[t], P->Tp_off[t]};
  }
  if ((st = upload(P->d_tdesc, tdesc, s)) != VTM_OK) return fail(st);
  {
    // tiles across the lines of each tile (for the dataflow sweeps)
    std::vector<int32_t> off(nparts + 1, 0), nb;
    std::vector<int32_t> seen(nparts, -1);
    for (int32_t t = 0; t < nparts; ++t) {
      for (int32_t q = P->port_off[t]; q < P->port_off[t + 1]; ++q) {
        const int32_t u = P->h_part[P->port_node[P->port_twin[q]]];
        if (u != t && seen[u] != t) {
          seen[u] = t;
          nb.push_back(u);
        }
      }
      off[t + 1] = (int32_t)nb.size();
    }
    if ((st = upload(P->d_nbr_off, off, s)) != VTM_OK) return fail(st);
    if ((st = upload(P->d_nbr, nb, s)) != VTM_OK) return fail(st);
  }
  if ((st = upload(P->d_port_loc, P->port_loc, s)) != VTM_OK) return fail(st);
  std::vector<int32_t> port_pos(P->port_node.size());
  for (size_t q = 0; q < port_pos.size(); ++q) port_pos[q] = P->iperm[P->port_node[q]];
  if ((st = upload(P->d_port_pos, port_pos, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->d_twin, P->port_twin, s)) != VTM_OK) return fail(st);
  if ((st = upload(P->d_run, P->port_run, s)) != VTM_OK) return fail(st);
  const size_t npt = std::max<size_t>(P->port_node.size(), 1);
  if ((st = dev_alloc(P->d_c64, npt * sizeof(double))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_state64, 4 * npt * sizeof(double))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_v, (size_t)n * sizeof(double))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_v2, (size_t)n * sizeof(double))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_xacc, (size_t)n * sizeof(double))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_r, (size_t)n * sizeof(double))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_bcol, (size_t)n * sizeof(double))) != VTM_OK) return fail(st);
  // two sweeps' worth (the one-warp-per-tile sweeps reduce one while writing the next)
  if ((st = dev_alloc(P->d_partials, 2 * sizeof(double) * std::max<size_t>(nparts, 4096))) != VTM_OK)
    return fail(st);
  // the control block, then one sweep counter per CTA of the one-warp-per-tile
  // kernels (their grids have at most one CTA per tile)
  if ((st = dev_alloc(P->d_ctrl, sizeof(SweepCtrl) + 4 * ((size_t)P->nparts + 4))) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_err, 64)) != VTM_OK) return fail(st);
  if ((st = dev_alloc(P->d_red, 256)) != VTM_OK) return fail(st);
  if (cudaMemsetAsync(P->d_red.p, 0, 256, s) != cudaSuccess) return fail(VTM_ECUDA);  // counters start at 0
  if (P->hist_cap == 0) {
    if ((st = dev_alloc(P->d_hist, 16)) != VTM_OK) return fail(st);
  }
  if (cudaMallocHost(&P->h_ctrl, sizeof(SweepCtrl)) != cudaSuccess) {
    P->h_ctrl = nullptr;
    return fail(VTM_ENOMEM);
  }
  if (cudaEventCreate(&P->ev0) != cudaSuccess || cudaEventCreate(&P->ev1) != cudaSuccess ||
      cudaEventCreate(&P->evs0) != cudaSuccess || cudaEventCreate(&P->evs1) != cudaSuccess)
    return fail(VTM_ECUDA);
  if ((st = assemble_local(P)) != VTM_OK) return fail(st);
  *out = P;
  return VTM_OK;
}

extern "C" vtm_status vtm_set_values(vtm_plan_t P, const double* vals) {
  if (!P || !vals) return VTM_EINVAL;
  std::vector<double> old = P->h_vals;
  vtm_status st = fetch(P->h_vals, vals, (size_t)P->nnz);
  if (st != VTM_OK) return st;
  for (double v : P->h_vals)
    if (!std::isfinite(v)) {
      P->h_vals = old;
      set_detail("vtm_set_values: non-finite value");
      return VTM_EINVAL;
    }
  if (P->symmetric) {
    for (int64_t i = 0; i < P->n; ++i)
      for (int64_t q = P->h_rowptr[i]; q < P->h_rowptr[i + 1]; ++q) {
        int32_t j = P->h_colidx[q];
        if (j <= i) continue;
        int64_t t = csr_find(P, j, (int32_t)i);
        if (t < 0 || P->h_vals[t] != P->h_vals[q]) {
          P->h_vals = old;
          set_detail("vtm_set_values: the plan was made for a symmetric matrix");
          return VTM_EINVAL;
        }
      }
  }
  // the torn lines and the lagged couplings must stay the same
  if (!same_cut_structure(P)) {
    P->h_vals = old;
    set_detail("vtm_set_values: the set of torn lines or lagged couplings changed");
    return VTM_EINVAL;
  }
  P->w_dirty = true;
  st = assemble_local(P);
  if (st != VTM_OK) {
    P->h_vals = old;
    P->w_dirty = true;
    assemble_local(P);
    return st;
  }
  VTM_CUDA_TRY(cudaMemcpyAsync(P->d_vals.p, P->h_vals.data(), P->nnz * sizeof(double),
                               cudaMemcpyHostToDevice, P->stream));
  VTM_CUDA_TRY(cudaStreamSynchronize(P->stream));
  P->factored = false;
  dev_free(P->d_vals_df);
  P->vals_df_state = 0;
  P->ell_state = 0;  // the ELL copy of A follows the values
  if (P->transposed) {
    vtm_destroy(P->transposed);
    P->transposed = nullptr;
  }
  return VTM_OK;
}

extern "C" vtm_status vtm_plan_get_stats(vtm_plan_t P, vtm_plan_stats* s) {
  if (!P || !s) return VTM_EINVAL;
  s->n = P->n;
  s->nparts = P->nparts;
  s->nports = (int64_t)P->port_node.size();
  s->nlagged = (int64_t)P->lag_i.size();
  s->sum_p2 = P->sum_p2;
  s->max_ports = P->max_ports;
  s->max_nodes = P->max_nodes;
  s->max_band = P->max_bw;
  s->symmetric = P->symmetric ? 1 : 0;
  s->t_bytes = (int64_t)(P->d_T64.bytes + P->d_T32.bytes + P->d_T16.bytes + P->d_E.bytes +
                         P->d_Tp32.bytes + P->d_Tp16.bytes + P->d_Tpdf.bytes);
  s->factor_bytes = (int64_t)(P->d_Lc.bytes + P->d_Uc.bytes);
  s->sweep_kernel = P->opts.method == VTM_METHOD_ASYNC   ? P->dataflow_kernel
                    : P->tuned_kernel[P->opts.precision] ? P->tuned_kernel[P->opts.precision]
                                                         : P->opts.sweep_kernel;
  s->sum_tri = P->sum_tri;
  s->packed_bytes = (int64_t)(P->d_Tp32.bytes + P->d_Tp16.bytes + P->d_Tpdf.bytes);
  s->batch_kernel = P->batch_used;
  return VTM_OK;
}

extern "C" vtm_status vtm_get_ports(vtm_plan_t P, int32_t* node, int32_t* remote, int32_t* part,
                                    int32_t* twin) {
  if (!P) return VTM_EINVAL;
  const size_t npt = P->port_node.size();
  for (size_t s = 0; s < npt; ++s) {
    if (node) node[s] = P->port_node[s];
    if (remote) remote[s] = P->port_remote[s];
    if (part) part[s] = P->h_part[P->port_node[s]];
    if (twin) twin[s] = P->port_twin[s];
  }
  return VTM_OK;
}

extern "C" void vtm_destroy(vtm_plan_t P) {
  if (!P) return;
  if (P->transposed) vtm_destroy(P->transposed);
  for (int i = 0; i < 4; ++i) {
    P->sweep_graph[i].reset();
    P->batch_graph[i].reset();
  }
  for (DevBuf* b : P->all_bufs()) dev_free(*b);
  if (P->h_ctrl) cudaFreeHost(P->h_ctrl);
  if (P->ev0) cudaEventDestroy(P->ev0);
  if (P->ev1) cudaEventDestroy(P->ev1);
  if (P->evs0) cudaEventDestroy(P->evs0);
  if (P->evs1) cudaEventDestroy(P->evs1);
  delete P;
}

extern "C" const char* vtm_strerror(vtm_status s) {
  switch (s) {
    case VTM_OK: return "success";
    case VTM_EINVAL: return "invalid argument";
    case VTM_ENOMEM: return "out of memory";
    case VTM_ESINGULAR: return "singular local matrix (bad pivot)";
    case VTM_ENOCONV: return "tolerance not reached within the sweep/refinement limit";
    case VTM_EDIVERGED: return "iteration diverged";
    case VTM_ETIMEOUT: return "device-side wait timed out";
    case VTM_ECUDA: return "CUDA runtime error";
    case VTM_EINTERNAL: return "internal error";
    case VTM_ENOTFACTORED: return "plan not factored";
  }
  return "unknown status";
}

extern "C" const char* vtm_last_error_detail(void) { return g_detail.c_str(); }
