// CG preconditioned by diagonal incomplete Cholesky (DIC), the preconditioner the
// paper names for its pressure CG (Sec. 2.6.1), on the symmetric LDU matrix.
//
// Cells are eliminated in the mesh's internal (RCM) numbering; since every
// internal face has owner < neighbour, the owner is the earlier cell:
//   d_i = D_i - sum_{f: N(f)=i} L_f^2 / d_O(f)                       (factor)
//   z = M^-1 r:  z_i = (r_i - sum_{f: N(f)=i} L_f z_O(f)) / d_i        (forward)
//                z_i -= (sum_{f: O(f)=i} L_f z_N(f)) / d_i             (backward)
// with M = (Dd + Lo) Dd^-1 (Dd + Lo^T).  Both recurrences run along dependency
// levels (level(i) = 1 + the largest level among the cells that i depends on),
// computed once per mesh on the host: one launch per level for the factor and
// per sweep, the backward sweep taking the levels in reverse order (every face
// joins cells of different levels).  On a 64^3 Kuhn mesh that is 437 levels of
// ~3,600 cells each, so an application costs ~870 dependent launches: the
// preconditioner is here for fidelity and comparison; the multigrid V-cycle is
// the fast one.
#include <algorithm>
#include <mutex>
#include <vector>

#include "krylov_common.cuh"

namespace difvm {

struct DicLevels {
  int nlev = 0;
  std::vector<int> ptr;     // [nlev + 1] host: cells of level l at cells[ptr[l] .. ptr[l+1])
  int* cells = nullptr;     // device, grouped by level, ascending inside a level
};

void dic_free(DicLevels* d) {
  if (!d) return;
  cudaFree(d->cells);
  delete d;
}

namespace {
std::mutex g_dic_mu;

difvm_status dic_levels(difvm_mesh* m, DicLevels** out) {
  std::lock_guard<std::mutex> lk(g_dic_mu);
  if (!m->dic) {
    std::vector<int2> on(std::max(m->ni, 1));
    if (m->ni > 0) DIFVM_CUDA(cudaMemcpy(on.data(), m->on, sizeof(int2) * m->ni, cudaMemcpyDeviceToHost));
    // faces are sorted by (owner, neighbour): a cell's owners (its dependencies)
    // all precede it, so one pass in face order settles every level
    std::vector<int> lev(m->nc, 0);
    for (int f = 0; f < m->ni; ++f) lev[on[f].y] = std::max(lev[on[f].y], lev[on[f].x] + 1);
    int nlev = 0;
    for (int i = 0; i < m->nc; ++i) nlev = std::max(nlev, lev[i] + 1);
    auto* d = new (std::nothrow) DicLevels();
    if (!d) return set_error(DIFVM_ENOMEM, "host allocation failed");
    d->nlev = nlev;
    d->ptr.assign(nlev + 1, 0);
    for (int i = 0; i < m->nc; ++i) d->ptr[lev[i] + 1]++;
    for (int l = 0; l < nlev; ++l) d->ptr[l + 1] += d->ptr[l];
    std::vector<int> fill(d->ptr.begin(), d->ptr.end() - 1), cells(m->nc);
    for (int i = 0; i < m->nc; ++i) cells[fill[lev[i]]++] = i;
    if (cudaMalloc(&d->cells, sizeof(int) * std::max(m->nc, 1)) != cudaSuccess ||
        cudaMemcpy(d->cells, cells.data(), sizeof(int) * m->nc, cudaMemcpyHostToDevice) != cudaSuccess) {
      dic_free(d);
      return set_error(DIFVM_ECUDA, "DIC level upload failed");
    }
    m->dic = d;
  }
  *out = m->dic;
  return DIFVM_OK;
}

constexpr int kDB = 256;

// d_i = D_i - sum over faces where i is the neighbour of L_f^2 / d_owner
template <typename T>
__global__ void k_dic_factor(int n, const int* cells, Topo t, const T* D, const T* L, T* d) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = cells[k];
  T s = D[i];
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e], f = ent >> 1;
    if (f >= t.ni) break;
    if (ent & 1) {
      const T l = L[f];
      s -= l * l / d[t.on[f].x];
    }
  }
  d[i] = s;
}

// forward sweep of one level: z_i = (r_i - sum_{i neighbour} L_f z_owner) / d_i
template <typename T>
__global__ void k_dic_fwd(int n, const int* cells, Topo t, const T* L, const T* d, const T* r, T* z,
                          const int* done) {
  if (*done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = cells[k];
  T s = r[i];
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e], f = ent >> 1;
    if (f >= t.ni) break;
    if (ent & 1) s -= L[f] * z[t.on[f].x];
  }
  z[i] = s / d[i];
}

// backward sweep of one level: z_i -= (sum_{i owner} L_f z_neighbour) / d_i
template <typename T>
__global__ void k_dic_bwd(int n, const int* cells, Topo t, const T* L, const T* d, T* z, const int* done) {
  if (*done) return;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int i = cells[k];
  T s = T(0);
  const int e1 = t.cptr[i + 1];
  for (int e = t.cptr[i]; e < e1; ++e) {
    const int ent = t.cent[e], f = ent >> 1;
    if (f >= t.ni) break;
    if (!(ent & 1)) s += L[f] * z[t.on[f].y];
  }
  z[i] -= s / d[i];
}

// r = b - A x; bb, rr; convergence at the start
template <typename T, int MW>
__global__ void __launch_bounds__(kKB) k_dcg_init(Topo t, Mat<T> A, const T* b, const T* x, T* r, KWork w) {
  const int nc = t.nc;
  DotAcc<T> bb, rr;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    T ax[1];
    spmv_row<T, 1, MW>(t, A, i, x, ax, 1u);
    const T bi = b[i], ri = bi - ax[0];
    r[i] = ri;
    bb.add(bi, bi);
    rr.add(ri, ri);
  }
  double v[2] = {bb.get(), rr.get()}, tot[2];
  if (!grid_sum<2>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.bb = tot[0];
  s.rr = tot[1];
  s.res0 = sqrt(s.rr);
  s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
  s.iters = 0;
  s.status = DIFVM_OK;
  s.zero_rhs = s.bb == 0.0;
  s.done = s.zero_rhs || s.rr <= s.tol2;
  if (!isfinite(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
}

template <typename T>
__global__ void k_dcg_zero(int nc, T* x, KWork w) {
  if (!w.st[0].zero_rhs) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) x[i] = T(0);
}

// x += alpha p; r -= alpha q; rr and the convergence test
template <typename T>
__global__ void __launch_bounds__(kKB) k_dcg_update(int nc, const T* p, const T* q, T* x, T* r, KWork w) {
  if (w.st[0].done) return;
  const T al = (T)w.st[0].alpha;
  DotAcc<T> rr;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    x[i] += al * p[i];
    const T ri = r[i] - al * q[i];
    r[i] = ri;
    rr.add(ri, ri);
  }
  double v[1] = {rr.get()}, tot[1];
  if (!grid_sum<1>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.iters += 1;
  s.rr = tot[0];
  if (!isfinite(s.rr) || !isfinite(s.alpha)) { s.done = 1; s.status = DIFVM_ENONFINITE; return; }
  if (s.rr <= s.tol2) { s.done = 1; return; }
  if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; }
}

// r.z; beta = rz / rz_previous (first: rz only)
template <typename T>
__global__ void __launch_bounds__(kKB) k_dcg_rz(int nc, const T* r, const T* z, KWork w, int first) {
  if (w.st[0].done) return;
  DotAcc<T> rz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) rz.add(r[i], z[i]);
  double v[1] = {rz.get()}, tot[1];
  if (!grid_sum<1>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.beta = first ? 0.0 : tot[0] / s.rz;
  s.rz = tot[0];
}

// p = z + beta p (first: p = z)
template <typename T>
__global__ void __launch_bounds__(kKB) k_dcg_p(int nc, const T* z, T* p, KWork w, int first) {
  if (w.st[0].done) return;
  const T be = (T)w.st[0].beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] + be * p[i];
}

__global__ void k_dcg_info(const KState* st, difvm_solve_info* info) {
  if (threadIdx.x != 0) return;
  difvm_solve_info o;
  o.iters = st->iters;
  o.refinements = 0;
  o.status = st->status;
  o.pad = 0;
  o.res0 = st->res0;
  o.res = sqrt(st->rr);
  o.bnorm = sqrt(st->bb);
  *info = o;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

struct DicLayout {
  size_t val, r, p, q, z, d, st, part, ticket, total;
};
DicLayout dic_layout(const difvm_mesh* m, size_t e, int G) {
  DicLayout L{};
  size_t o = 0;
  auto take = [&](size_t b) { size_t r = o; o += up256(std::max<size_t>(b, 1)); return r; };
  L.val = take((size_t)std::max<int64_t>(m->ell_nslots, 1) * e);
  L.r = take((size_t)m->nc * e);
  L.p = take((size_t)m->nc * e);
  L.q = take((size_t)m->nc * e);
  L.z = take((size_t)m->nc * e);
  L.d = take((size_t)m->nc * e);
  L.st = take(sizeof(KState));
  L.part = take((size_t)G * kMaxParts * sizeof(double));
  L.ticket = take(256);
  L.total = o;
  return L;
}
int dic_grid(const difvm_mesh* m) { return std::max(1, std::min((int)blocks_for(m->nc, kKB), m->num_sms * 4)); }
}  // namespace

size_t dic_workspace_bytes(difvm_mesh* m, size_t elt) {
  DicLevels* d = nullptr;
  if (dic_levels(m, &d) != DIFVM_OK) return 0;
  return dic_layout(m, elt, dic_grid(m)).total;
}

template <typename T, int MW>
static difvm_status dic_solve_mw(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo,
                                 const T* b, T* x, void* ws, size_t wsbytes, difvm_solve_info* info,
                                 cudaStream_t st) {
  DicLevels* DL = nullptr;
  DIFVM_TRY(dic_levels(m, &DL));
  const int G = dic_grid(m), nc = m->nc;
  const DicLayout Ly = dic_layout(m, sizeof(T), G);
  if (!ws || wsbytes < Ly.total)
    return set_error(DIFVM_EINVAL, "workspace of %zu bytes < %zu needed (DIC)", wsbytes, Ly.total);
  char* W = (char*)ws;
  T *val = (T*)(W + Ly.val), *r = (T*)(W + Ly.r), *p = (T*)(W + Ly.p), *q = (T*)(W + Ly.q);
  T *z = (T*)(W + Ly.z), *d = (T*)(W + Ly.d);
  KWork w;
  w.st = (KState*)(W + Ly.st);
  w.part = (double*)(W + Ly.part);
  w.ticket = (unsigned*)(W + Ly.ticket);
  w.maxit = o->max_iter > 0 ? o->max_iter : 1000;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  const Topo t = m->topo();
  if (m->ell_nslots > 0) {
    k_ell_fill<T><<<blocks_for(m->ell_nslots, 256), 256, 0, st>>>((int)m->ell_nslots, m->ell_map, Lo, Lo, val);
    DIFVM_TRY(check_launch("ell_fill"));
  }
  const Mat<T> A{D, m->ell(), val};
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), st));
  const int* done = &w.st[0].done;
  // factor, level by level
  for (int l = 0; l < DL->nlev; ++l) {
    const int n = DL->ptr[l + 1] - DL->ptr[l];
    k_dic_factor<T><<<blocks_for(n, kDB), kDB, 0, st>>>(n, DL->cells + DL->ptr[l], t, D, Lo, d);
    count_launch();
  }
  DIFVM_TRY(check_error("dic_factor"));
  auto apply = [&](cudaStream_t s) {   // z = M^-1 r
    for (int l = 0; l < DL->nlev; ++l) {
      const int n = DL->ptr[l + 1] - DL->ptr[l];
      k_dic_fwd<T><<<blocks_for(n, kDB), kDB, 0, s>>>(n, DL->cells + DL->ptr[l], t, Lo, d, r, z, done);
    }
    for (int l = DL->nlev - 1; l >= 0; --l) {
      const int n = DL->ptr[l + 1] - DL->ptr[l];
      k_dic_bwd<T><<<blocks_for(n, kDB), kDB, 0, s>>>(n, DL->cells + DL->ptr[l], t, Lo, d, z, done);
    }
    for (int l = 0; l < 2 * DL->nlev; ++l) count_launch();
  };
  k_dcg_init<T, MW><<<G, kKB, 0, st>>>(t, A, b, x, r, w);
  k_dcg_zero<T><<<G, kKB, 0, st>>>(nc, x, w);
  DIFVM_TRY(check_launch("dcg_init"));
  count_launch();
  apply(st);
  k_dcg_rz<T><<<G, kKB, 0, st>>>(nc, r, z, w, 1);
  k_dcg_p<T><<<G, kKB, 0, st>>>(nc, z, p, w, 1);
  DIFVM_TRY(check_launch("dcg_p"));
  count_launch();
  auto iter = [&](cudaStream_t s) {
    k_pcg_spmv<T, 1, MW><<<G, kKB, 0, s>>>(t, A, p, q, w);
    k_dcg_update<T><<<G, kKB, 0, s>>>(nc, p, q, x, r, w);
    apply(s);
    k_dcg_rz<T><<<G, kKB, 0, s>>>(nc, r, z, w, 0);
    k_dcg_p<T><<<G, kKB, 0, s>>>(nc, z, p, w, 0);
    count_launch(); count_launch(); count_launch(); count_launch();
  };
  int* counter = reinterpret_cast<int*>(w.ticket) + 1;
  const bool graph = stream_capturing(st);
  if (graph) {
    DIFVM_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    WhileLoop Lw;
    DIFVM_TRY(while_open(st, Lw));
    iter(Lw.side);
    k_loop_cond<<<1, 32, 0, Lw.side>>>(done_flags(w.st), kStateInts, 1, counter, w.maxit + 2, Lw.h);
    difvm_status e = check_launch("loop_cond");
    DIFVM_TRY(while_close(Lw));
    DIFVM_TRY(e);
  } else {
    const int chunk = o->check_every > 0 ? o->check_every : 8;
    KState hs;
    for (int it = 0; it < w.maxit + chunk; it += chunk) {
      for (int k = 0; k < chunk; ++k) iter(st);
      DIFVM_TRY(check_error("dcg_iter"));
      DIFVM_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
      DIFVM_CUDA(cudaStreamSynchronize(st));
      if (hs.done) break;
    }
  }
  if (info) {
    k_dcg_info<<<1, 32, 0, st>>>(w.st, info);
    DIFVM_TRY(check_launch("dcg_info"));
  }
  if (graph) return DIFVM_OK;
  KState hs;
  DIFVM_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  return (difvm_status)hs.status;
}

template <typename T>
difvm_status dic_solve(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo, const T* b, T* x,
                       void* ws, size_t wsbytes, difvm_solve_info* info, cudaStream_t st) {
  if (m->ell_wmax <= 4) return dic_solve_mw<T, 4>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
  if (m->ell_wmax <= 8) return dic_solve_mw<T, 8>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
  return dic_solve_mw<T, 0>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
}
template difvm_status dic_solve<float>(difvm_mesh*, const difvm_solve_opts*, const float*, const float*,
                                       const float*, float*, void*, size_t, difvm_solve_info*, cudaStream_t);
template difvm_status dic_solve<double>(difvm_mesh*, const difvm_solve_opts*, const double*, const double*,
                                        const double*, double*, void*, size_t, difvm_solve_info*, cudaStream_t);

}  // namespace difvm
