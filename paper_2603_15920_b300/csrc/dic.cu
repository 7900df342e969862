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
// computed once per mesh on the host; the backward sweep takes the levels in
// reverse order (every face joins cells of different levels).  On a 64^3 Kuhn
// mesh that is 437 levels of ~3,600 cells each.  Each sweep (and the factor) is
// one launch whose rows wait on the rows they depend on (see the single-launch
// sweeps below); the same sweeps apply DILU, the non-symmetric form, to the
// momentum BiCGStab.  The chain of 437 dependent levels remains: the
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

}  // namespace

// ------------------------------------------------ single-launch level sweeps
// The factor and the two triangular sweeps of DIC / DILU in one launch each,
// instead of one launch per dependency level.  Rows are taken in level order
// (the cells array: levels ascending; the backward sweep walks it from the
// end): each warp claims the next 32 positions from a ticket, and a row waits
// for the rows it depends on (the face partners of lower level) by polling
// their ready flags, then computes and publishes its own flag.  A row's
// dependencies come earlier in the order, so they were claimed by warps that
// are already running: every wait ends (lanes of one warp may wait on each
// other across a level boundary; independent thread scheduling lets them
// progress).  A row loads its dependencies' indices and coefficients before it
// waits.  Each wait is bounded (about 4M polls); one that runs out marks the
// solver states DIFVM_ETIMEOUT and the row proceeds, so the launch always ends.
// Flags hold the sweep's epoch (a counter bumped before every sweep), so they
// need clearing once per solve only.  The sums run in CSR order, as in the
// per-level kernels, so the results are the same bit for bit.
struct SweepCtl {
  unsigned epoch, ticket;
};
constexpr int kSB = 256;

__global__ void k_sweep_begin(SweepCtl* c) {
  c->epoch += 1u;
  c->ticket = 0u;
}

__device__ __forceinline__ unsigned ld_acq(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_rel(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_rlx(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// wait until row j is ready (relaxed polls, then one acquire fence); false if
// the wait ran out
__device__ __forceinline__ bool sweep_wait(const unsigned* flag, int j, unsigned epoch) {
  if (ld_acq(flag + j) == epoch) return true;
  for (int k = 0; k < (1 << 22); ++k) {
    if (ld_rlx(flag + j) == epoch) {
      asm volatile("fence.acq_rel.gpu;" ::: "memory");
      return true;
    }
  }
  return false;
}

// MODE 0: factor d_i = D_i - sum_{f: N(f)=i} L_f U_f / d_O(f)
// MODE 1: forward z_i = (r_i - sum_{f: N(f)=i} L_f z_O(f)) / d_i     (NC components)
// MODE 2: backward z_i -= (sum_{f: O(f)=i} U_f z_N(f)) / d_i
template <typename T, int NC, int MODE>
__global__ void __launch_bounds__(kSB) k_ilu_sweep(int nc, const int* __restrict__ order, Topo t,
                                                   const T* __restrict__ D, const T* __restrict__ L,
                                                   const T* __restrict__ U, T* d, const T* r, T* z,
                                                   unsigned* flag, const SweepCtl* ctl, KState* st, int nst) {
  if (MODE != 0) {   // a Krylov apply after every component converged: nothing to do
    bool all = true;
    for (int c = 0; c < nst; ++c) all = all && st[c].done;
    if (all) return;
  }
  const unsigned epoch = ctl->epoch;
  unsigned* ticket = const_cast<unsigned*>(&ctl->ticket);
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (;;) {
    unsigned cl = 0;
    if (lane == 0) cl = atomicAdd(ticket, 1u);
    cl = __shfl_sync(0xffffffffu, cl, 0);
    const long long k = (long long)cl * 32 + lane;
    if ((long long)cl * 32 >= nc) break;
    if (k < nc) {
      const int i = order[MODE == 2 ? nc - 1 - (int)k : (int)k];
      const int e0 = t.cptr[i], e1 = t.cptr[i + 1];
      // the row's dependencies (face partners eliminated before it) and their
      // coefficients, loaded before any wait; rows of more than kDep such
      // partners take the rest in a second pass
      constexpr int kDep = 6;
      int jd[kDep];
      T cd[kDep];
      int nd = 0, e = e0;
      for (; e < e1 && nd < kDep; ++e) {
        const int ent = t.cent[e], f = ent >> 1;
        if (f >= t.ni) break;
        const bool dep = MODE == 2 ? !(ent & 1) : (ent & 1);
        if (!dep) continue;
        const int2 on = t.on[f];
        jd[nd] = MODE == 2 ? on.y : on.x;
        cd[nd] = MODE == 0 ? L[f] * U[f] : (MODE == 1 ? L[f] : U[f]);
        ++nd;
      }
      T s[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) s[c] = T(0);
      if (MODE == 0) s[0] = D[i];
      if (MODE == 1)
#pragma unroll
        for (int c = 0; c < NC; ++c) s[c] = r[c * nc + i];
      for (int q = 0; q < nd; ++q) ok = sweep_wait(flag, jd[q], epoch) && ok;
      for (int q = 0; q < nd; ++q) {
        if (MODE == 0) s[0] -= cd[q] / __ldcg(d + jd[q]);
        else if (MODE == 1)
#pragma unroll
          for (int c = 0; c < NC; ++c) s[c] -= cd[q] * __ldcg(z + c * nc + jd[q]);
        else
#pragma unroll
          for (int c = 0; c < NC; ++c) s[c] += cd[q] * __ldcg(z + c * nc + jd[q]);
      }
      for (; e < e1; ++e) {   // rows with more partners than kDep
        const int ent = t.cent[e], f = ent >> 1;
        if (f >= t.ni) break;
        const bool dep = MODE == 2 ? !(ent & 1) : (ent & 1);
        if (!dep) continue;
        const int2 on = t.on[f];
        const int j = MODE == 2 ? on.y : on.x;
        ok = sweep_wait(flag, j, epoch) && ok;
        if (MODE == 0) s[0] -= L[f] * U[f] / __ldcg(d + j);
        else if (MODE == 1)
#pragma unroll
          for (int c = 0; c < NC; ++c) s[c] -= L[f] * __ldcg(z + c * nc + j);
        else
#pragma unroll
          for (int c = 0; c < NC; ++c) s[c] += U[f] * __ldcg(z + c * nc + j);
      }
      if (MODE == 0) {
        d[i] = s[0];
      } else if (MODE == 1) {
        const T di = d[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c * nc + i] = s[c] / di;
      } else {
        const T di = d[i];
#pragma unroll
        for (int c = 0; c < NC; ++c) z[c * nc + i] -= s[c] / di;
      }
      st_rel(flag + i, epoch);   // release: the row's results are visible before its flag
    }
  }
  if (!ok)
    for (int c = 0; c < nst; ++c) {
      st[c].status = DIFVM_ETIMEOUT;
      st[c].done = 1;
    }
}

// workspace of the sweeps: the factor d, the ready flags, the control words
size_t ilu_extra_bytes(const difvm_mesh* m, size_t elt) {
  return (((size_t)m->nc * elt + 255) / 256 + ((size_t)m->nc * 4 + 255) / 256 + 1) * 256;
}
struct IluWs {
  char* d;
  unsigned* flag;
  SweepCtl* ctl;
};
IluWs ilu_ws(const difvm_mesh* m, size_t elt, char* extra) {
  const size_t a = ((size_t)m->nc * elt + 255) / 256 * 256, b = ((size_t)m->nc * 4 + 255) / 256 * 256;
  return IluWs{extra, (unsigned*)(extra + a), (SweepCtl*)(extra + a + b)};
}
// one block per SM: more resident warps only poll further ahead of the front
// (measured on the 64^3 Kuhn pressure matrix: 5.1 ms per DIC-CG iteration with
// one block per SM, 5.6 ms with eight; sleeping between polls was slower)
int sweep_grid(const difvm_mesh* m) {
  return std::max(1, std::min((int)blocks_for(m->nc, kSB), m->num_sms));
}

// d of the DILU (U != L) or DIC (U == L) factor in the mesh's internal order
template <typename T>
difvm_status ilu_factor(difvm_mesh* m, const T* D, const T* L, const T* U, char* extra, KState* st, int nst,
                        cudaStream_t s) {
  DicLevels* DL = nullptr;
  DIFVM_TRY(dic_levels(m, &DL));
  const IluWs w = ilu_ws(m, sizeof(T), extra);
  DIFVM_CUDA(cudaMemsetAsync(w.flag, 0, (size_t)m->nc * 4, s));
  DIFVM_CUDA(cudaMemsetAsync(w.ctl, 0, sizeof(SweepCtl), s));
  k_sweep_begin<<<1, 1, 0, s>>>(w.ctl);
  k_ilu_sweep<T, 1, 0><<<sweep_grid(m), kSB, 0, s>>>(m->nc, DL->cells, m->topo(), D, L, U ? U : L, (T*)w.d,
                                                      nullptr, nullptr, w.flag, w.ctl, st, nst);
  count_launch();
  return check_launch("ilu_factor");
}

// z = M^-1 r for ncomp components (r, z: [ncomp][nc]); skipped once st[0..nst) are done
template <typename T>
difvm_status ilu_apply(difvm_mesh* m, int ncomp, const T* L, const T* U, char* extra, const T* r, T* z,
                       KState* st, int nst, cudaStream_t s) {
  DicLevels* DL = m->dic;
  const IluWs w = ilu_ws(m, sizeof(T), extra);
  const int G = sweep_grid(m);
  const Topo t = m->topo();
  const T* Uu = U ? U : L;
  k_sweep_begin<<<1, 1, 0, s>>>(w.ctl);
  switch (ncomp) {
    case 1: k_ilu_sweep<T, 1, 1><<<G, kSB, 0, s>>>(m->nc, DL->cells, t, nullptr, L, Uu, (T*)w.d, r, z, w.flag, w.ctl, st, nst); break;
    case 2: k_ilu_sweep<T, 2, 1><<<G, kSB, 0, s>>>(m->nc, DL->cells, t, nullptr, L, Uu, (T*)w.d, r, z, w.flag, w.ctl, st, nst); break;
    default: k_ilu_sweep<T, 3, 1><<<G, kSB, 0, s>>>(m->nc, DL->cells, t, nullptr, L, Uu, (T*)w.d, r, z, w.flag, w.ctl, st, nst); break;
  }
  k_sweep_begin<<<1, 1, 0, s>>>(w.ctl);
  switch (ncomp) {
    case 1: k_ilu_sweep<T, 1, 2><<<G, kSB, 0, s>>>(m->nc, DL->cells, t, nullptr, L, Uu, (T*)w.d, r, z, w.flag, w.ctl, st, nst); break;
    case 2: k_ilu_sweep<T, 2, 2><<<G, kSB, 0, s>>>(m->nc, DL->cells, t, nullptr, L, Uu, (T*)w.d, r, z, w.flag, w.ctl, st, nst); break;
    default: k_ilu_sweep<T, 3, 2><<<G, kSB, 0, s>>>(m->nc, DL->cells, t, nullptr, L, Uu, (T*)w.d, r, z, w.flag, w.ctl, st, nst); break;
  }
  for (int k = 0; k < 3; ++k) count_launch();
  return check_launch("ilu_apply");
}
template difvm_status ilu_factor<float>(difvm_mesh*, const float*, const float*, const float*, char*, KState*, int,
                                        cudaStream_t);
template difvm_status ilu_factor<double>(difvm_mesh*, const double*, const double*, const double*, char*, KState*,
                                         int, cudaStream_t);
template difvm_status ilu_apply<float>(difvm_mesh*, int, const float*, const float*, char*, const float*, float*,
                                       KState*, int, cudaStream_t);
template difvm_status ilu_apply<double>(difvm_mesh*, int, const double*, const double*, char*, const double*,
                                        double*, KState*, int, cudaStream_t);

namespace {

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
  size_t val, r, p, q, z, st, part, ticket, extra, total;
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
  L.st = take(sizeof(KState));
  L.part = take((size_t)G * kMaxParts * sizeof(double));
  L.ticket = take(256);
  L.extra = take(ilu_extra_bytes(m, e));   // factor, ready flags, sweep control
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
  T* z = (T*)(W + Ly.z);
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
  DIFVM_TRY(ilu_factor<T>(m, D, Lo, Lo, W + Ly.extra, w.st, 1, st));
  auto apply = [&](cudaStream_t s) {   // z = M^-1 r
    ilu_apply<T>(m, 1, Lo, Lo, W + Ly.extra, r, z, w.st, 1, s);
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
