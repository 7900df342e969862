// Aggregation multigrid preconditioner for the symmetric pressure system
// (the CG of Sec. 2.6.1).
//
// The paper preconditions CG with ILU; an incomplete factorisation is applied
// by two triangular solves whose dependency chains run through every RCM level
// of the mesh, which leaves a 148-SM GPU idle.  Here the preconditioner is one
// V-cycle of aggregation multigrid, whose every step is a data-parallel sweep:
//
//   hierarchy (once per mesh, host): cells are paired along their strongest
//     face (largest c_f = |S|^2/(S.d)), a cell left alone joins its strongest
//     neighbour's pair; two such passes make one level (about 4-5 cells per
//     aggregate), down to at most kAmgCoarsest cells;
//   operators (every solve, device): Galerkin products with piecewise-constant
//     prolongation, i.e. sums of the finer level's coefficients (a coarse
//     diagonal is the sum of its cells' diagonals plus twice the coefficients
//     of the faces inside it; a coarse face coefficient is the sum of the fine
//     faces between its two aggregates), each sum in a fixed order;
//   V-cycle: two Jacobi sweeps with Chebyshev weights before and after the
//     coarse correction, which is scaled by kAmgScale; the coarsest level
//     solved with a dense inverse (Gauss-Jordan in one block, FP32, symmetrised);
//   mixed precision: CG with FP64 accuracy (float-float vectors) around the FP32
//     V-cycle (no refinement sweeps).
//
// The V-cycle is a fixed symmetric positive-definite linear operator, so CG
// keeps its guarantees; it changes the iteration count, not the solution.
#include <algorithm>
#include <mutex>
#include <numeric>
#include <vector>

#include "krylov_common.cuh"

namespace difvm {

// Jacobi weights of the two smoothing sweeps: the reciprocals of the degree-2
// Chebyshev nodes on [1/2, 2] (Gershgorin bounds the spectrum of D^-1 A of these
// diagonally dominant matrices by 2), 5/4 -+ (3/4) cos(pi/4).  The two sweeps
// before the coarse correction use (w1, w2), the two after it (w2, w1): the
// smoother is the degree-2 Chebyshev polynomial in D^-1 A either way, so the
// V-cycle stays symmetric.  CPU prototype on a 40^3 Kuhn mesh: 22 CG iterations
// against 25 with two omega = 0.7 sweeps, at the same cost per iteration.
constexpr double kAmgW1 = 1.0 / (1.25 + 0.75 * 0.70710678118654752);
constexpr double kAmgW2 = 1.0 / (1.25 - 0.75 * 0.70710678118654752);
// over-correction of the coarse-grid correction (64^3 Kuhn cavity with the
// Chebyshev-weighted sweeps: 22 CG iterations at 1.9 against 23 at 1.8 and 24 at 2.0)
constexpr double kAmgScale = 1.9;
// the first Jacobi iterate from zero, w1 rD r, rounded twice and never fused into
// a following add: the restriction stores it for the coarse level's
// pre-smoothing, and every kernel that forms it on the fly gets the same number
__device__ __forceinline__ float amg_x1(float rD, float r) { return __fmul_rn(__fmul_rn((float)kAmgW1, rD), r); }
__device__ __forceinline__ double amg_x1(double rD, double r) { return __dmul_rn(__dmul_rn(kAmgW1, rD), r); }
// a prolongated value y + s xc (coarse correction scaled by kAmgScale), one
// explicit fma, so that a stored and an on-the-fly prolongation agree
__device__ __forceinline__ float amg_prol(float y, float xc) { return __fmaf_rn((float)kAmgScale, xc, y); }
__device__ __forceinline__ double amg_prol(double y, double xc) { return __fma_rn(kAmgScale, xc, y); }
constexpr int kAmgCoarsest = 192;   // coarsen until at most this many cells (6 x 32)
constexpr int kAmgMaxLevels = 16;
constexpr int kAB = 256;            // threads per block of the AMG kernels
constexpr int kAmgCoarseTB = 256;   // threads per block of the coarsest solve (8 rows a block)
constexpr int kAmgBigLevel = 100000;   // from this size a level's sweeps are bandwidth-bound
// levels of at most this many rows store their residual in child order (its
// scattered stores stay in L2): 64^3 cavity 14.90 -> 14.75 ms per step; with the
// 12.6M-row mesh level of a 128^3 cavity or a 15.8M-row batch it was slower
constexpr int kAmgChildOrderRows = 4 << 20;

// One level as the kernels see it.  Level 0 is the mesh (its SpMV uses the
// sliced ELL); on coarser levels `on` / `cptr` / `cent` hold the level's own
// faces.  The restriction fields describe the map to the next level.
struct AmgLev {
  int n, nf;
  const int2* on;
  const int* cptr;
  const int* cent;                    // entries F<<1|side, ascending F per cell
  // levels >= 1: sliced ELL of the off-diagonal entries (slices of 32 rows,
  // slot = soff[i/32] + 32 k + i%32, k in CSR order; padding: column i, face -1)
  const int* soff;
  const int* ecol;
  const int* eface;
  int nslots;
  const int* agg;                     // [n] cell -> next-level cell
  const int* eagg;                    // [slots of the level's ELL] agg of the slot's column
  const int *ch_ptr, *ch_idx;         // next-level cell -> its cells
  const int* cpos;                    // [n] position of the cell in ch_idx (the inverse map)
  const int *ci_ptr, *ci_idx;         // next-level cell -> faces inside it
  const int *cf_ptr, *cf_idx;         // next-level face -> faces mapped to it
};

struct AmgHier {
  int nlev = 0;
  std::vector<AmgLev> lev;
  std::vector<void*> allocs;
  // launch shape per level: lanes per row of the level's sweeps, lanes per
  // aggregate of its restriction into the next level (the defaults of
  // amg_default_lanes, or what amg_tune measured fastest)
  std::vector<int> tpr, rl;
};

void amg_free(AmgHier* h) {
  if (!h) return;
  for (void* p : h->allocs) cudaFree(p);
  delete h;
}

// ------------------------------------------------------------ hierarchy (host)
namespace {

struct Graph {
  int n = 0;
  std::vector<int2> on;     // faces, (I, J) with I < J, ascending
  std::vector<double> w;    // face weights
};

// one pairwise pass: agg[i] in [0, na)
void pair_pass(const Graph& g, std::vector<int>& agg, int& na) {
  const int nf = (int)g.on.size();
  std::vector<int> ord(nf);
  std::iota(ord.begin(), ord.end(), 0);
  std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return g.w[a] > g.w[b]; });
  agg.assign(g.n, -1);
  na = 0;
  for (int f : ord) {
    const int I = g.on[f].x, J = g.on[f].y;
    if (agg[I] < 0 && agg[J] < 0) agg[I] = agg[J] = na++;
  }
  std::vector<int> best(g.n, -1);  // strongest neighbour
  for (int f : ord) {
    const int I = g.on[f].x, J = g.on[f].y;
    if (best[I] < 0) best[I] = J;
    if (best[J] < 0) best[J] = I;
  }
  for (int i = 0; i < g.n; ++i) {
    if (agg[i] >= 0) continue;
    const int j = best[i];
    agg[i] = (j >= 0 && agg[j] >= 0) ? agg[j] : na++;
  }
}

// coarse graph of an aggregation; fmap[f] = coarse face, or -1 inside an aggregate
void coarse_graph(const Graph& g, const std::vector<int>& agg, int na, Graph& c, std::vector<int>& fmap) {
  const int nf = (int)g.on.size();
  std::vector<int64_t> key(nf, -1);
  std::vector<int64_t> keys;
  keys.reserve(nf);
  for (int f = 0; f < nf; ++f) {
    int a = agg[g.on[f].x], b = agg[g.on[f].y];
    if (a == b) continue;
    if (a > b) std::swap(a, b);
    key[f] = (int64_t)a * na + b;
    keys.push_back(key[f]);
  }
  std::sort(keys.begin(), keys.end());
  keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
  c.n = na;
  c.on.resize(keys.size());
  c.w.assign(keys.size(), 0.0);
  for (size_t k = 0; k < keys.size(); ++k) c.on[k] = make_int2((int)(keys[k] / na), (int)(keys[k] % na));
  fmap.assign(nf, -1);
  for (int f = 0; f < nf; ++f) {
    if (key[f] < 0) continue;
    const int F = (int)(std::lower_bound(keys.begin(), keys.end(), key[f]) - keys.begin());
    fmap[f] = F;
    c.w[F] += g.w[f];
  }
}

template <typename T>
difvm_status upload_vec(AmgHier* H, const T** dst, const std::vector<T>& v) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(v.size(), 1) * sizeof(T);
  DIFVM_CUDA(cudaMalloc(&p, bytes));
  H->allocs.push_back(p);
  if (!v.empty()) DIFVM_CUDA(cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  *dst = (const T*)p;
  return DIFVM_OK;
}

// CSR of `key[i]` (values in [0, nk)) listing i ascending
void group_by(const std::vector<int>& key, int nk, std::vector<int>& ptr, std::vector<int>& idx,
              const std::vector<char>* keep = nullptr) {
  ptr.assign(nk + 1, 0);
  for (size_t i = 0; i < key.size(); ++i)
    if (key[i] >= 0 && (!keep || (*keep)[i])) ptr[key[i] + 1]++;
  for (int k = 0; k < nk; ++k) ptr[k + 1] += ptr[k];
  idx.assign(ptr[nk], 0);
  std::vector<int> fill(ptr.begin(), ptr.end() - 1);
  for (size_t i = 0; i < key.size(); ++i)
    if (key[i] >= 0 && (!keep || (*keep)[i])) idx[fill[key[i]]++] = (int)i;
}

// Relabel the cells of a new level so that, inside windows of 256 ids, they come
// in decreasing number of faces: the 32-row slices of the level's sliced ELL
// then hold rows of similar length (padding ~45% -> ~8% on Kuhn meshes), while
// ids stay within their window (locality kept).  agg (finer cell -> new cell)
// and fmap (finer face -> new face) follow; the new level's faces are re-sorted.
void relabel_by_degree(Graph& g, std::vector<int>& agg, std::vector<int>& fmap) {
  const int n = g.n, nf = (int)g.on.size();
  std::vector<int> deg(n, 0);
  for (const int2& o : g.on) { deg[o.x]++; deg[o.y]++; }
  std::vector<int> order(n), newid(n);
  std::iota(order.begin(), order.end(), 0);
  for (int w0 = 0; w0 < n; w0 += 256) {
    const int w1 = std::min(n, w0 + 256);
    std::stable_sort(order.begin() + w0, order.begin() + w1, [&](int a, int b) { return deg[a] > deg[b]; });
  }
  for (int k = 0; k < n; ++k) newid[order[k]] = k;
  for (int& a : agg) a = newid[a];
  std::vector<int64_t> key(nf);
  for (int F = 0; F < nf; ++F) {
    int a = newid[g.on[F].x], b = newid[g.on[F].y];
    if (a > b) std::swap(a, b);
    key[F] = (int64_t)a * n + b;
  }
  std::vector<int> fo(nf), fnew(nf);
  std::iota(fo.begin(), fo.end(), 0);
  std::sort(fo.begin(), fo.end(), [&](int a, int b) { return key[a] < key[b]; });
  Graph h;
  h.n = n;
  h.on.resize(nf);
  h.w.resize(nf);
  for (int k = 0; k < nf; ++k) {
    const int F = fo[k];
    fnew[F] = k;
    h.on[k] = make_int2((int)(key[F] / n), (int)(key[F] % n));
    h.w[k] = g.w[F];
  }
  for (int& F : fmap)
    if (F >= 0) F = fnew[F];
  g = std::move(h);
}

difvm_status build_hier(difvm_mesh* m, AmgHier* H) {
  // level-0 graph: the mesh's internal faces weighted by c_f
  Graph g;
  g.n = m->nc;
  g.on.resize(m->ni);
  if (m->ni > 0) DIFVM_CUDA(cudaMemcpy(g.on.data(), m->on, sizeof(int2) * m->ni, cudaMemcpyDeviceToHost));
  std::vector<V4<double>> ck(m->ni);
  if (m->ni > 0) DIFVM_CUDA(cudaMemcpy(ck.data(), m->ck64, sizeof(V4<double>) * m->ni, cudaMemcpyDeviceToHost));
  g.w.resize(m->ni);
  for (int f = 0; f < m->ni; ++f) g.w[f] = ck[f].x;

  std::vector<int> ecol_host;   // the current level's ELL columns (level 0: the mesh's ELL)
  ecol_host.resize(std::max<int64_t>(m->ell_nslots, 0));
  if (m->ell_nslots > 0)
    DIFVM_CUDA(cudaMemcpy(ecol_host.data(), m->ell_col, sizeof(int) * m->ell_nslots, cudaMemcpyDeviceToHost));
  while (true) {
    AmgLev L{};
    L.n = g.n;
    L.nf = (int)g.on.size();
    const int lvl = (int)H->lev.size();
    if (lvl == 0) {
      L.on = m->on;
      L.cptr = m->cptr;
      L.cent = m->cent;
    } else {
      DIFVM_TRY(upload_vec(H, &L.on, g.on));
      std::vector<int> cptr(g.n + 1, 0), cent(2 * g.on.size());
      for (const int2& o : g.on) { cptr[o.x + 1]++; cptr[o.y + 1]++; }
      for (int i = 0; i < g.n; ++i) cptr[i + 1] += cptr[i];
      std::vector<int> fill(cptr.begin(), cptr.end() - 1);
      for (int f = 0; f < (int)g.on.size(); ++f) {   // ascending face id per cell
        cent[fill[g.on[f].x]++] = f << 1;
        cent[fill[g.on[f].y]++] = (f << 1) | 1;
      }
      const int nsl = (g.n + 31) / 32;
      std::vector<int> soff(nsl + 1, 0);
      for (int sl = 0; sl < nsl; ++sl) {
        int w = 0;
        for (int i = 32 * sl; i < std::min(g.n, 32 * sl + 32); ++i) w = std::max(w, cptr[i + 1] - cptr[i]);
        soff[sl + 1] = soff[sl] + 32 * w;
      }
      std::vector<int> ecol(std::max(soff[nsl], 1)), eface(std::max(soff[nsl], 1), -1);
      for (int i = 0; i < g.n; ++i) {
        const int sl = i >> 5, w = (soff[sl + 1] - soff[sl]) / 32;
        for (int k = 0; k < w; ++k) {
          const int slot = soff[sl] + 32 * k + (i & 31);
          const int e = cptr[i] + k;
          if (e < cptr[i + 1]) {
            const int2 o = g.on[cent[e] >> 1];
            ecol[slot] = (cent[e] & 1) ? o.x : o.y;
            eface[slot] = cent[e] >> 1;
          } else {
            ecol[slot] = i;
          }
        }
      }
      L.nslots = soff[nsl];
      ecol_host = ecol;
      DIFVM_TRY(upload_vec(H, &L.cptr, cptr));
      DIFVM_TRY(upload_vec(H, &L.cent, cent));
      DIFVM_TRY(upload_vec(H, &L.soff, soff));
      DIFVM_TRY(upload_vec(H, &L.ecol, ecol));
      DIFVM_TRY(upload_vec(H, &L.eface, eface));
    }
    const bool last = g.n <= kAmgCoarsest || lvl + 1 >= kAmgMaxLevels;
    if (!last) {
      // two pairwise passes make the next level
      std::vector<int> a1, a2, f1, f2;
      int n1, n2;
      Graph g1, g2;
      pair_pass(g, a1, n1);
      coarse_graph(g, a1, n1, g1, f1);
      pair_pass(g1, a2, n2);
      coarse_graph(g1, a2, n2, g2, f2);
      if (n2 > 0.85 * g.n) {   // coarsening stalled: this is the coarsest level
        H->lev.push_back(L);
        break;
      }
      std::vector<int> agg(g.n), fmap(g.on.size()), inside(g.on.size(), -1);
      for (int i = 0; i < g.n; ++i) agg[i] = a2[a1[i]];
      for (size_t f = 0; f < g.on.size(); ++f) {
        const int F1 = f1[f];
        fmap[f] = F1 < 0 ? -1 : f2[F1];
      }
      relabel_by_degree(g2, agg, fmap);
      for (size_t f = 0; f < g.on.size(); ++f)
        if (fmap[f] < 0) inside[f] = agg[g.on[f].x];
      std::vector<int> chp, chi, cip, cii, cfp, cfi;
      group_by(agg, n2, chp, chi);
      group_by(inside, n2, cip, cii);
      group_by(fmap, (int)g2.on.size(), cfp, cfi);
      DIFVM_TRY(upload_vec(H, &L.agg, agg));
      std::vector<int> eagg(ecol_host.size());
      for (size_t k = 0; k < ecol_host.size(); ++k) eagg[k] = agg[ecol_host[k]];
      DIFVM_TRY(upload_vec(H, &L.eagg, eagg));
      DIFVM_TRY(upload_vec(H, &L.ch_ptr, chp));
      DIFVM_TRY(upload_vec(H, &L.ch_idx, chi));
      std::vector<int> cpos(g.n);
      for (size_t c = 0; c < chi.size(); ++c) cpos[chi[c]] = (int)c;
      DIFVM_TRY(upload_vec(H, &L.cpos, cpos));
      DIFVM_TRY(upload_vec(H, &L.ci_ptr, cip));
      DIFVM_TRY(upload_vec(H, &L.ci_idx, cii));
      DIFVM_TRY(upload_vec(H, &L.cf_ptr, cfp));
      DIFVM_TRY(upload_vec(H, &L.cf_idx, cfi));
      H->lev.push_back(L);
      g = std::move(g2);
      continue;
    }
    H->lev.push_back(L);
    break;
  }
  H->nlev = (int)H->lev.size();
  return DIFVM_OK;
}

std::mutex g_amg_mu;

}  // namespace

void amg_default_lanes(AmgHier* H);
void amg_tune(difvm_mesh* m, AmgHier* H);

difvm_status amg_hier(difvm_mesh* m, AmgHier** out) {
  std::lock_guard<std::mutex> lk(g_amg_mu);
  if (!m->amg) {
    AmgHier* H = new (std::nothrow) AmgHier();
    if (!H) return set_error(DIFVM_ENOMEM, "host allocation failed");
    difvm_status s = build_hier(m, H);
    if (s != DIFVM_OK) {
      amg_free(H);
      return s;
    }
    amg_default_lanes(H);
    if (m->autotune) amg_tune(m, H);
    m->amg = H;
  }
  *out = m->amg;
  return DIFVM_OK;
}

// the mesh's autotune mode changed: 0 puts the default launch shapes back, 2
// measures them again (a hierarchy not built yet is tuned when it is built)
void amg_retune(difvm_mesh* m, int mode) {
  std::lock_guard<std::mutex> lk(g_amg_mu);
  if (!m->amg) return;
  if (mode == 0) amg_default_lanes(m->amg);
  else if (mode == 2) amg_tune(m, m->amg);
}

// ---------------------------------------------------------- workspace layout
// [ELL values | r p q z | per level: D rD L E r s a b | coarsest inverse | states | partials |
//  tickets | flags | fused-level descriptors | barrier]; a batched mesh has one state and
//  one ticket per case
struct AmgLayout {
  size_t val, vec[4], D[kAmgMaxLevels], rD[kAmgMaxLevels], L[kAmgMaxLevels], E[kAmgMaxLevels],
      r[kAmgMaxLevels], s[kAmgMaxLevels], a[kAmgMaxLevels], b[kAmgMaxLevels], inv, st, part, ticket, flag, tail,
      bar, total;
};

static size_t up256a(size_t b) { return (b + 255) / 256 * 256; }

// the CG kernels and the level-0 sweep with r.z: grid-stride, one wave (their
// grid reductions finish once instead of once per wave of blocks)
static int amg_grid(const difvm_mesh* m) {
  return std::max(1, std::min((int)blocks_for(m->nc, kKB), m->num_sms * 4));
}

static AmgLayout amg_layout(const difvm_mesh* m, const AmgHier* H, size_t e) {
  AmgLayout A{};
  size_t o = 0;
  auto take = [&](size_t bytes) { size_t r = o; o += up256a(std::max<size_t>(bytes, 1)); return r; };
  A.val = take((size_t)std::max<int64_t>(m->ell_nslots, 1) * e);
  for (int k = 0; k < 4; ++k) A.vec[k] = take((size_t)m->nc * e);
  for (int l = 0; l < H->nlev; ++l) {
    const AmgLev& L = H->lev[l];
    A.D[l] = take((size_t)L.n * e);
    A.rD[l] = take((size_t)L.n * e);
    A.L[l] = take((size_t)L.nf * e);
    A.E[l] = take((size_t)(l > 0 ? L.nslots : 1) * e);   // sliced-ELL values (levels >= 1)
    A.r[l] = take((size_t)L.n * e);
    A.s[l] = take((size_t)(l > 0 ? L.n : 1) * e);       // w1 rD r of a coarse level's r
    A.a[l] = take((size_t)L.n * e);
    A.b[l] = take((size_t)L.n * e);
  }
  const int nco = H->lev[H->nlev - 1].n;
  A.inv = take((size_t)nco * nco * sizeof(float));
  A.st = take((size_t)(m->seg ? m->ncases : 4) * sizeof(KState));
  // partials: one per block of the CG kernels and of the level-0 smoothing with
  // r.z (batched: one per block of the segmented CG kernels)
  const size_t nblk = m->seg ? std::max(amg_grid(m), m->seg_nblk) : amg_grid(m);
  A.part = take(nblk * kMaxParts * sizeof(double));
  A.ticket = take((size_t)(m->seg ? m->ncases : 2) * sizeof(unsigned));
  A.flag = take(4 * sizeof(int));
  A.tail = take(kAmgMaxLevels * 256);   // level descriptors of the fused coarse-level kernel
  A.bar = take(128);                     // its grid barrier's arrival counter
  A.total = o;
  return A;
}

size_t amg_workspace_bytes(difvm_mesh* m, size_t elt) {
  AmgHier* H = nullptr;
  if (amg_hier(m, &H) != DIFVM_OK) return 0;
  // + the float-float x, r (low part), p, q of the mixed-precision form
  return amg_layout(m, H, elt).total + 7 * up256a((size_t)m->nc * 4);
}

// ------------------------------------------------------------------ kernels
template <typename T>
__global__ void k_amg_rd(int n, const T* D, T* rD) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) rD[i] = T(1) / D[i];
}

// coarse diagonal: sum of the cells' diagonals + twice the faces inside
template <typename T>
__global__ void k_amg_diag(int n1, AmgLev L, const T* D, const T* Lv, T* D1, T* rD1) {
  int K = blockIdx.x * blockDim.x + threadIdx.x;
  if (K >= n1) return;
  T d = T(0);
  for (int c = L.ch_ptr[K]; c < L.ch_ptr[K + 1]; ++c) d += D[L.ch_idx[c]];
  for (int c = L.ci_ptr[K]; c < L.ci_ptr[K + 1]; ++c) d += T(2) * Lv[L.ci_idx[c]];
  D1[K] = d;
  rD1[K] = T(1) / d;
}

// coarse face coefficient: sum of the fine faces between the two aggregates
template <typename T>
__global__ void k_amg_faces(int nf1, AmgLev L, const T* Lv, T* L1) {
  int F = blockIdx.x * blockDim.x + threadIdx.x;
  if (F >= nf1) return;
  T s = T(0);
  for (int c = L.cf_ptr[F]; c < L.cf_ptr[F + 1]; ++c) s += Lv[L.cf_idx[c]];
  L1[F] = s;
}

// sliced-ELL values of a coarse level from its face coefficients (0 on padding)
template <typename T>
__global__ void k_amg_entries(int nslots, const int* eface, const T* Lv, T* E) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nslots) return;
  const int f = eface[k];
  E[k] = f < 0 ? T(0) : Lv[f];
}

// dense inverse of the coarsest matrix (SPD: Gauss-Jordan without pivoting), one
// block, in FP32 (the B300's FP64 rate is about 1/64 of FP32 and this runs on one
// SM), then symmetrised; it serves only as the preconditioner's coarsest solve
template <typename T>
__global__ void __launch_bounds__(512) k_amg_dense_inv(AmgLev L, const T* D, const T* Lv, float* A) {
  // thread (ty, tx) of a 16 x 32 grid owns the elements (ty + 16a, tx + 32b),
  // a < 12, b < 6: a 12 x 6 register tile (512 threads leave 128 registers each)
  constexpr int NR = kAmgCoarsest / 16, NC = kAmgCoarsest / 32;
  const int n = L.n;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k] = 0.f;
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) A[i * n + i] = (float)D[i];
  for (int f = threadIdx.x; f < L.nf; f += blockDim.x) {
    const int2 o = L.on[f];
    A[o.x * n + o.y] = (float)Lv[f];
    A[o.y * n + o.x] = (float)Lv[f];
  }
  __syncthreads();
  float a[NR][NC];
#pragma unroll
  for (int p = 0; p < NR; ++p)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const int i = ty + 16 * p, j = tx + 32 * q;
      a[p][q] = (i < n && j < n) ? A[i * n + j] : 0.f;
    }
  __shared__ float row[kAmgCoarsest], col[kAmgCoarsest];
  for (int k = 0; k < n; ++k) {
    // row k and column k (before the step) to shared memory: every tile element
    // is visited with a compile-time index, predicated on being in row/column k
#pragma unroll
    for (int p = 0; p < NR; ++p)
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const int i = ty + 16 * p, j = tx + 32 * q;
        if (i == k && j < n) row[j] = a[p][q];
        if (j == k && i < n) col[i] = a[p][q];
      }
    __syncthreads();
    const float rp = 1.f / row[k];
    float rj[NC], ci[NR];
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const int j = tx + 32 * q;
      rj[q] = (j == k) ? rp : row[j < n ? j : 0] * rp;
    }
#pragma unroll
    for (int p = 0; p < NR; ++p) {
      const int i = ty + 16 * p;
      ci[p] = col[i < n ? i : 0];
    }
#pragma unroll
    for (int p = 0; p < NR; ++p) {
      const bool rowk = ty + 16 * p == k;
#pragma unroll
      for (int q = 0; q < NC; ++q) {
        const bool colk = tx + 32 * q == k;
        const float old = colk ? 0.f : a[p][q];
        a[p][q] = rowk ? rj[q] : old - ci[p] * rj[q];
      }
    }
    __syncthreads();
  }
  // write back symmetrised: the exact inverse is symmetric
#pragma unroll
  for (int p = 0; p < NR; ++p)
#pragma unroll
    for (int q = 0; q < NC; ++q) {
      const int i = ty + 16 * p, j = tx + 32 * q;
      if (i < n && j < n) A[i * n + j] = a[p][q];
    }
  __syncthreads();
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) {
    const int i = t / n, j = t - i * n;
    if (i < j) {
      const float v = 0.5f * (A[i * n + j] + A[j * n + i]);
      A[i * n + j] = v;
      A[j * n + i] = v;
    }
  }
}

// (A x)_i of row i.  TPR == 1: level 0, one thread per row, the mesh's ELL.
// TPR > 1: a coarser level's sliced ELL, TPR lanes per row (lane t takes
// slots t, t + TPR, ..., two in flight per pass), so the dependent loads of a
// row (slice offset, column, gathered value) take a few round trips whatever
// its width; the lanes are summed by a fixed xor tree and every lane gets the
// total.  x is a functor so that smoothed values can be formed on the fly.
// `ok` = the row exists; all lanes of a warp must call it (shuffles).
// PROL: x takes (column, its aggregate), the aggregates coming from L.eagg
// in the same slot order, so that a prolongated value needs no dependent load.
template <bool PROL, class XF>
__device__ __forceinline__ auto xat(XF& x, int c, int a) {
  if constexpr (PROL) return x(c, a);
  else return x(c);
}
template <typename T, int TPR, bool PROL = false, class XF>
__device__ __forceinline__ T lev_row(const Mat<T>& A, const AmgLev& L, const T* D, const T* Lv, int i, int t,
                                     bool ok, XF x) {
  if constexpr (TPR == 1) {
    if (!ok) return T(0);
    T y = __ldg(A.D + i) * xat<PROL>(x, i, PROL ? __ldg(L.agg + i) : 0);
    if (A.E.W == 4) {
      const int4 j4 = ell_cols4(A.E, i);
      const int4 g4 = PROL ? __ldg(reinterpret_cast<const int4*>(L.eagg) + i) : make_int4(0, 0, 0, 0);
      T a[4];
      Vec4Load<T>::get(A.val, i, a);
      y += a[0] * xat<PROL>(x, j4.x, g4.x);
      y += a[1] * xat<PROL>(x, j4.y, g4.y);
      y += a[2] * xat<PROL>(x, j4.z, g4.z);
      y += a[3] * xat<PROL>(x, j4.w, g4.w);
      return y;
    }
    int base, step, w;
    ell_row(A.E, i, base, step, w);
    for (int k = 0; k < w; ++k) {
      const int o = base + step * k;
      y += __ldg(A.val + o) * xat<PROL>(x, __ldg(A.E.col + o), PROL ? __ldg(L.eagg + o) : 0);
    }
    return y;
  } else {
    // a lane's first Q slots: all column and value loads, then all gathers,
    // then the sums in slot order (three dependent round trips for rows of up
    // to Q * TPR slots); longer rows continue two slots per pass
    constexpr int Q = (TPR >= 8 ? 32 : 16) / TPR;
    T y = T(0);
    if (ok) {
      const int o0 = __ldg(L.soff + (i >> 5));
      const int w = (__ldg(L.soff + (i >> 5) + 1) - o0) >> 5;
      const int ob = o0 + (i & 31) + 32 * t;
      const T xi = t == 0 ? xat<PROL>(x, i, PROL ? __ldg(L.agg + i) : 0) : T(0);
      int c[Q], ag[Q];
      T v[Q], xv[Q];
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const bool in = t + q * TPR < w;
        c[q] = in ? __ldg(L.ecol + ob + 32 * q * TPR) : -1;
        ag[q] = in && PROL ? __ldg(L.eagg + ob + 32 * q * TPR) : 0;
        v[q] = in ? Lv[ob + 32 * q * TPR] : T(0);   // Lv: ELL values
      }
#pragma unroll
      for (int q = 0; q < Q; ++q) xv[q] = c[q] >= 0 ? xat<PROL>(x, c[q], ag[q]) : T(0);
      if (t == 0) y = D[i] * xi;
#pragma unroll
      for (int q = 0; q < Q; ++q) y += v[q] * xv[q];
      int k = t + Q * TPR, o = ob + 32 * Q * TPR;
      for (; k + TPR < w; k += 2 * TPR, o += 64 * TPR) {
        const int c0 = __ldg(L.ecol + o), c1 = __ldg(L.ecol + o + 32 * TPR);
        const int a0 = PROL ? __ldg(L.eagg + o) : 0, a1 = PROL ? __ldg(L.eagg + o + 32 * TPR) : 0;
        const T v0 = Lv[o], v1 = Lv[o + 32 * TPR];
        const T x0 = xat<PROL>(x, c0, a0), x1 = xat<PROL>(x, c1, a1);
        y += v0 * x0;
        y += v1 * x1;
      }
      if (k < w) y += Lv[o] * xat<PROL>(x, __ldg(L.ecol + o), PROL ? __ldg(L.eagg + o) : 0);
    }
#pragma unroll
    for (int d = TPR / 2; d > 0; d >>= 1) y += __shfl_xor_sync(0xffffffffu, y, d);
    return y;
  }
}

// pre-smoothing from zero, two sweeps: x1 = w1 rD r, y = x1 + w2 rD (r - A x1).
// PS: x1 comes in formed (sr, written with r by the restriction), so a column
// costs one gather instead of two.
template <typename T, int TPR, bool PS>
__global__ void __launch_bounds__(kAB) k_amg_pre(AmgLev L, Mat<T> A, const T* D, const T* rD, const T* Lv,
                                                 const T* r, const T* sr, T* y, const int* done) {
  pdl_chain();
  if (*done) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, i = g / TPR, t = g % TPR;
  const bool ok = i < L.n;
  const T w2 = (T)kAmgW2;
  auto x1 = [&](int j) { return PS ? sr[j] : amg_x1(rD[j], r[j]); };
  const T ax = lev_row<T, TPR>(A, L, D, Lv, i, t, ok, x1);
  if (ok && t == 0) y[i] = x1(i) + w2 * rD[i] * (r[i] - ax);
}

// residual after pre-smoothing: res = r - A y.  CO: stored in child order (row
// i at cpos[i]) so that the restriction sums each aggregate's children from one
// contiguous range; the scattered stores pay off while the level's residual
// stays in L2 (kAmgChildOrderRows)
template <typename T, int TPR, bool CO>
__global__ void __launch_bounds__(kAB) k_amg_resid(AmgLev L, Mat<T> A, const T* D, const T* Lv, const T* r,
                                                   const T* y, T* res, const int* done) {
  pdl_chain();
  if (*done) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, i = g / TPR, t = g % TPR;
  const bool ok = i < L.n;
  const int pos = CO ? (ok && t == 0 ? __ldg(L.cpos + i) : 0) : i;
  auto xy = [&](int j) { return y[j]; };
  const T ay = lev_row<T, TPR>(A, L, D, Lv, i, t, ok, xy);
  if (ok && t == 0) res[pos] = r[i] - ay;
}

// restriction: rc_K = sum of res over the cells of K, and sc_K = w1 rD_K rc_K
// (the coarse level's first Jacobi iterate, for its pre-smoothing).  RL == 1:
// one thread per K, four children in flight; RL > 1: RL lanes per K, each
// summing its children in ascending order, then a fixed xor tree.
template <typename T, int RL, bool CO>
__global__ void __launch_bounds__(kAB) k_amg_restrict(int n1, AmgLev L, const T* res, T* rc, const T* rD1,
                                                      T* sc, const int* done) {
  pdl_chain();
  if (*done) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, K = g / RL, t = g % RL;
  T s = T(0);
  if (K < n1) {   // CO: res in child order, the children of K are res[ch_ptr[K] .. ch_ptr[K+1])
    auto at = [&](int c) { return CO ? res[c] : res[L.ch_idx[c]]; };
    const int c1 = L.ch_ptr[K + 1];
    int c = L.ch_ptr[K] + t;
    if (RL == 1) {
      for (; c + 4 <= c1; c += 4) {
        const T r0 = at(c), r1 = at(c + 1), r2 = at(c + 2), r3 = at(c + 3);
        s += r0;
        s += r1;
        s += r2;
        s += r3;
      }
    }
    for (; c < c1; c += RL) s += at(c);
  }
#pragma unroll
  for (int d = RL / 2; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (K < n1 && t == 0) {
    rc[K] = s;
    sc[K] = amg_x1(rD1[K], s);
  }
}

// coarse correction and the first post-smoothing sweep: z = y + s P xc, out =
// z + w rD (r - A z).  PZ: y already holds z (k_amg_prol ran), a plain sweep;
// else z is formed on the fly from the per-slot aggregates.
template <typename T, int TPR, bool PZ>
__global__ void __launch_bounds__(kAB) k_amg_post1(AmgLev L, Mat<T> A, const T* D, const T* rD, const T* Lv,
                                                   const T* r, const T* y, const T* xc, T* out,
                                                   const int* done) {
  pdl_chain();
  if (*done) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, i = g / TPR, t = g % TPR;
  const bool ok = i < L.n;
  const T w = (T)kAmgW2;   // first sweep after the correction: w2
  if (PZ) {
    auto z = [&](int j) { return y[j]; };
    const T az = lev_row<T, TPR>(A, L, D, Lv, i, t, ok, z);
    if (ok && t == 0) out[i] = y[i] + w * rD[i] * (r[i] - az);
  } else {
    auto z = [&](int j, int a) { return amg_prol(y[j], xc[a]); };
    const T az = lev_row<T, TPR, true>(A, L, D, Lv, i, t, ok, z);
    if (ok && t == 0) out[i] = z(i, L.agg[i]) + w * rD[i] * (r[i] - az);
  }
}

// the coarse correction in place, y = y + s P xc (one thread per row), for a
// large level, whose corrected sweep then gathers one value per column
template <typename T>
__global__ void __launch_bounds__(kAB) k_amg_prol(AmgLev L, const T* xc, T* y, const int* done) {
  pdl_chain();
  if (*done) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < L.n) y[i] = amg_prol(y[i], xc[__ldg(L.agg + i)]);
}

// second post-smoothing sweep: v = u + w1 rD (r - A u)
template <typename T, int TPR>
__global__ void __launch_bounds__(kAB) k_amg_post2(AmgLev L, Mat<T> A, const T* D, const T* rD, const T* Lv,
                                                   const T* r, const T* u, T* v, const int* done) {
  pdl_chain();
  if (*done) return;
  const int g = blockIdx.x * blockDim.x + threadIdx.x, i = g / TPR, t = g % TPR;
  const bool ok = i < L.n;
  const T om = (T)kAmgW1;
  auto xu = [&](int j) { return u[j]; };
  const T au = lev_row<T, TPR>(A, L, D, Lv, i, t, ok, xu);
  if (ok && t == 0) v[i] = u[i] + om * rD[i] * (r[i] - au);
}

// the same sweep on level 0 of a CG iteration (grid-stride), also forming
// r.v: the last block sets beta (first = 1: rz only).  FP32: four blocks per SM
// (32 registers; 40 without the bound) so that the grid of 4 x SMs blocks runs
// in one wave.
template <typename T>
__global__ void __launch_bounds__(kKB, sizeof(T) == 4 ? 4 : 0) k_amg_post2_dot(AmgLev L, Mat<T> A, const T* rD, const T* r, const T* u,
                                                       T* v, KWork w, int first) {
  pdl_chain();
  if (w.st[0].done) return;
  const T om = (T)kAmgW1;
  DotAcc<T> rz;
  auto xu = [&](int j) { return u[j]; };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < L.n; i += gridDim.x * blockDim.x) {
    const T vi = u[i] + om * rD[i] * (r[i] - lev_row<T, 1>(A, L, nullptr, nullptr, i, 0, true, xu));
    v[i] = vi;
    rz.add(r[i], vi);
  }
  double tv[1] = {rz.get()}, tot[1];
  if (!grid_sum<1>(w, tv, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.beta = first ? 0.0 : tot[0] / s.rz;
  s.rz = tot[0];
}

// r.z and beta when the hierarchy has a single level (no smoothing kernel to fuse it into)
template <typename T>
__global__ void __launch_bounds__(kKB) k_apcg_rz(int nc, const T* r, const T* z, KWork w, int first) {
  if (w.st[0].done) return;
  DotAcc<T> rz;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) rz.add(r[i], z[i]);
  double v[1] = {rz.get()}, tot[1];
  if (!grid_sum<1>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.beta = first ? 0.0 : tot[0] / s.rz;
  s.rz = tot[0];
}

// coarsest level: x = A^{-1} r (dense inverse), one warp per row, eight rows a
// block: each block stages r in shared memory, each lane's at most
// kAmgCoarsest/32 entries of its row are loaded together, then a shuffle tree
// sums the lanes in a fixed order
template <typename T>
__global__ void __launch_bounds__(kAmgCoarseTB) k_amg_coarse(int n, const float* Ainv, const T* r, T* x,
                                                            const int* done) {
  pdl_chain();
  if (*done) return;
  constexpr int NJ = kAmgCoarsest / 32;
  __shared__ float rs[kAmgCoarsest];
  for (int j = threadIdx.x; j < n; j += blockDim.x) rs[j] = (float)r[j];
  __syncthreads();
  const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int i = blockIdx.x * nw + (threadIdx.x >> 5); i < n; i += gridDim.x * nw) {
    float a[NJ];
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      const int j = lane + 32 * q;
      a[q] = j < n ? Ainv[i * n + j] : 0.f;
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      const int j = lane + 32 * q;
      s += a[q] * (j < n ? rs[j] : 0.f);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[i] = (T)s;
  }
}

// -------------------------------------------- fused coarse levels (one launch)
// On request (difvm_mesh_amg_config), levels of fewer than a given number of
// rows, and the coarsest dense solve, run in one cooperative kernel: every
// pre-smoothing, residual, restriction, dense solve and post-smoothing sweep
// of those levels is a phase of the whole grid, phases separated by a grid
// barrier, instead of one launch per sweep.  The phases compute exactly what
// the per-level kernels compute, in the same order per row.  (Measured slower
// than the per-level kernels on the B300, hence off by default: see
// amg_tail_plan.)
constexpr int kTB = 512;            // threads per block of the fused kernel
constexpr int kTailMaxLev = kAmgMaxLevels;

// one level as the fused kernel sees it (a copy lives in the workspace)
template <typename T> struct TailLev {
  AmgLev L;
  const T *D, *rD, *Lv;   // diagonal, its reciprocal, sliced-ELL values
  T *r, *y, *u;           // right-hand side; work vectors (y ends as the output)
  int tpr, rl;            // lanes per row of the sweeps; per aggregate of the restriction
};
static_assert(sizeof(TailLev<double>) <= 256 && sizeof(TailLev<float>) <= 256 &&
                  sizeof(TailLev<double>) % sizeof(int) == 0 && sizeof(TailLev<float>) % sizeof(int) == 0,
              "a level descriptor must fit its 256-byte workspace slot, in whole ints");
template <typename T> struct TailArgs {
  const TailLev<T>* lev;  // [nlev]: the first fused level .. the coarsest
  int nlev;
  const float* Ainv;      // coarsest dense inverse
  const int* done;        // the CG (or every case of a batch) has converged
  unsigned* bar;          // the grid barrier's words (see tail_barrier)
  KState* st;             // solver states, marked ETIMEOUT if a barrier wait runs out
  int nst;
  int* all_done;          // batched solves: the all-cases-converged flag, or null
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier of a cooperative launch (every block resident): one arrival
// counter that only grows.  Every launch passes the same number of barriers,
// nbar, so the counter is a multiple of nbar G (G = blocks) when a launch starts
// (no block can pass the first barrier before all have arrived, so at most G - 1
// arrivals are ahead of a block that reads it then): base = the counter at the
// start rounded down to that multiple, and barrier k completes when the counter
// reaches base + (k + 1) G.  A block's thread 0 arrives with a release add and
// waits with acquire loads, at most ~4M polls (about a second); a wait that runs
// out returns false in every thread of its block (the solve is then closed with
// DIFVM_ETIMEOUT, and the counter is cleared before the next solve).
struct TailBar {
  unsigned* ctr;
  unsigned next;   // the counter value that completes the next barrier
};
__device__ __forceinline__ TailBar tail_bar_start(unsigned* ctr, unsigned nbar) {
  const unsigned G = gridDim.x, span = (nbar > 0 ? nbar : 1u) * G;
  const unsigned c = threadIdx.x == 0 ? ld_acquire_u32(ctr) : 0u;   // only thread 0 waits
  return TailBar{ctr, c - c % span + G};
}
__device__ __forceinline__ bool tail_barrier(TailBar& b) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int ok = 1;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(b.ctr) : "memory");
    int spins = 0;
    while ((int)(ld_acquire_u32(b.ctr) - b.next) < 0) {
      if (++spins > (1 << 22)) {
        ok = 0;
        break;
      }
    }
    ok_s = ok;
  }
  b.next += gridDim.x;
  __syncthreads();
  return ok_s != 0;
}

// Phases: grid-stride loops over whole warps of TPR-lane rows.  Vectors the
// kernel itself writes (r, y, u of the fused levels) are read through L2
// (__ldcg), since another block may have written them in the previous phase.
template <typename T, int TPR, class F>
__device__ __forceinline__ void tail_rows(int n, F&& body) {
  const int nvt = (int)(((int64_t)n * TPR + 31) & ~(int64_t)31);
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nvt; g += gridDim.x * blockDim.x)
    body(g / TPR, g % TPR);
}

template <typename T, int TPR>
__device__ void tail_pre(const TailLev<T>& P) {
  const T w2 = (T)kAmgW2;
  const Mat<T> A{};
  tail_rows<T, TPR>(P.L.n, [&](int i, int t) {
    const bool ok = i < P.L.n;
    auto x1 = [&](int j) { return amg_x1(P.rD[j], __ldcg(P.r + j)); };
    const T ax = lev_row<T, TPR>(A, P.L, P.D, P.Lv, i, t, ok, x1);
    if (ok && t == 0) P.y[i] = x1(i) + w2 * P.rD[i] * (__ldcg(P.r + i) - ax);
  });
}
template <typename T, int TPR>
__device__ void tail_resid(const TailLev<T>& P) {
  const Mat<T> A{};
  tail_rows<T, TPR>(P.L.n, [&](int i, int t) {
    const bool ok = i < P.L.n;
    auto xy = [&](int j) { return __ldcg(P.y + j); };
    const T ay = lev_row<T, TPR>(A, P.L, P.D, P.Lv, i, t, ok, xy);
    if (ok && t == 0) P.u[i] = __ldcg(P.r + i) - ay;
  });
}
template <typename T, int RL>
__device__ void tail_restrict(const TailLev<T>& P, int n1, T* rc) {
  tail_rows<T, RL>(n1, [&](int K, int t) {
    T s = T(0);
    if (K < n1) {
      const int c1 = P.L.ch_ptr[K + 1];
      for (int c = P.L.ch_ptr[K] + t; c < c1; c += RL) s += __ldcg(P.u + P.L.ch_idx[c]);
    }
#pragma unroll
    for (int d = RL / 2; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if (K < n1 && t == 0) rc[K] = s;
  });
}
template <typename T, int TPR>
__device__ void tail_post1(const TailLev<T>& P, const T* xc) {
  const T w = (T)kAmgW2;
  const Mat<T> A{};
  tail_rows<T, TPR>(P.L.n, [&](int i, int t) {
    const bool ok = i < P.L.n;
    auto z = [&](int j, int a) { return amg_prol(__ldcg(P.y + j), __ldcg(xc + a)); };
    const T az = lev_row<T, TPR, true>(A, P.L, P.D, P.Lv, i, t, ok, z);
    if (ok && t == 0) P.u[i] = z(i, P.L.agg[i]) + w * P.rD[i] * (__ldcg(P.r + i) - az);
  });
}
template <typename T, int TPR>
__device__ void tail_post2(const TailLev<T>& P) {
  const T om = (T)kAmgW1;
  const Mat<T> A{};
  tail_rows<T, TPR>(P.L.n, [&](int i, int t) {
    const bool ok = i < P.L.n;
    auto xu = [&](int j) { return __ldcg(P.u + j); };
    const T au = lev_row<T, TPR>(A, P.L, P.D, P.Lv, i, t, ok, xu);
    if (ok && t == 0) P.y[i] = __ldcg(P.u + i) + om * P.rD[i] * (__ldcg(P.r + i) - au);
  });
}
// coarsest level: y = A^{-1} r, one warp per row, lanes summed by a fixed tree
template <typename T>
__device__ void tail_coarse(const TailLev<T>& P, const float* Ainv) {
  constexpr int NJ = kAmgCoarsest / 32;
  const int n = P.L.n, lane = threadIdx.x & 31;
  const int wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  for (int i = wg; i < n; i += nw) {
    float a[NJ], x[NJ];
#pragma unroll
    for (int q = 0; q < NJ; ++q) {
      const int j = lane + 32 * q;
      a[q] = j < n ? Ainv[i * n + j] : 0.f;
      x[q] = j < n ? (float)__ldcg(P.r + j) : 0.f;
    }
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < NJ; ++q) s += a[q] * x[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) P.y[i] = (T)s;
  }
}

#define DIFVM_TAIL_TPR(tpr, F, ...) \
  do {                              \
    if ((tpr) == 2) F<T, 2>(__VA_ARGS__); \
    else if ((tpr) == 4) F<T, 4>(__VA_ARGS__); \
    else F<T, 8>(__VA_ARGS__);      \
  } while (0)

template <typename T>
__global__ void __launch_bounds__(kTB, 2) k_amg_tail(TailArgs<T> P) {
  if (*P.done) return;
  // the level descriptors, staged once in shared memory
  __shared__ __align__(16) TailLev<T> lev[kTailMaxLev];
  {
    const int nw = P.nlev * (int)(sizeof(TailLev<T>) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(P.lev);
    int* dst = reinterpret_cast<int*>(lev);
    for (int k = threadIdx.x; k < nw; k += blockDim.x) dst[k] = src[k];
  }
  __syncthreads();
  const int nl = P.nlev;
  TailBar bar = tail_bar_start(P.bar, 5u * (unsigned)(nl - 1));   // the barriers below, per launch
  bool ok = true;
  for (int k = 0; k + 1 < nl && ok; ++k) {   // down: smooth, residual, restrict
    const TailLev<T>& L = lev[k];
    DIFVM_TAIL_TPR(L.tpr, tail_pre, L);
    if (!(ok = tail_barrier(bar))) break;
    DIFVM_TAIL_TPR(L.tpr, tail_resid, L);
    if (!(ok = tail_barrier(bar))) break;
    if (L.rl == 1) tail_restrict<T, 1>(L, lev[k + 1].L.n, lev[k + 1].r);
    else tail_restrict<T, 8>(L, lev[k + 1].L.n, lev[k + 1].r);
    ok = tail_barrier(bar);
  }
  if (ok) {
    tail_coarse<T>(lev[nl - 1], P.Ainv);
    ok = nl == 1 || tail_barrier(bar);
  }
  for (int k = nl - 2; k >= 0 && ok; --k) {  // up: corrected sweep, second sweep
    const TailLev<T>& L = lev[k];
    DIFVM_TAIL_TPR(L.tpr, tail_post1, L, (const T*)lev[k + 1].y);
    if (!(ok = tail_barrier(bar))) break;
    DIFVM_TAIL_TPR(L.tpr, tail_post2, L);
    if (k > 0) ok = tail_barrier(bar);
  }
  if (!ok && threadIdx.x == 0) {
    for (int k = 0; k < P.nst; ++k) {
      P.st[k].status = DIFVM_ETIMEOUT;
      P.st[k].done = 1;
    }
    if (P.all_done) *P.all_done = 1;
  }
}
#undef DIFVM_TAIL_TPR

// copies the level descriptors into the workspace (a kernel, so that it also
// works under stream capture)
template <typename T> struct TailLevs { TailLev<T> lev[kTailMaxLev]; };
template <typename T>
__global__ void k_amg_tail_desc(TailLevs<T> d, int n, TailLev<T>* out) {
  for (int k = threadIdx.x; k < n; k += blockDim.x) out[k] = d.lev[k];
}

// --------------------------------------------------------------- CG kernels
// r = b - A x; bb, rr; convergence at the start; `gate` (may be null): when
// *gate != 0 the solve is closed at once (the outer refinement loop is done)
template <typename T, int MW>
__global__ void __launch_bounds__(kKB) k_apcg_init(Topo t, Mat<T> A, const T* b, T* x, T* r, KWork w,
                                                   const int* gate, int zero_x) {
  const int nc = t.nc;
  DotAcc<T> bb, rr;
  const bool skip = gate && *gate;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    if (skip) break;
    if (zero_x) x[i] = T(0);
    T ax[1];
    if (zero_x) ax[0] = T(0);
    else spmv_row<T, 1, MW>(t, A, i, x, ax, 1u);
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
  s.done = skip || s.zero_rhs || s.rr <= s.tol2;
  if (!skip && !isfinite(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
}

template <typename T>
__global__ void k_apcg_zero(int nc, T* x, KWork w) {
  if (!w.st[0].zero_rhs) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) x[i] = T(0);
}

// p = z + beta p (first: p = z)
template <typename T>
__global__ void __launch_bounds__(kKB) k_apcg_p(int nc, const T* z, T* p, KWork w, int first) {
  pdl_chain();
  if (w.st[0].done) return;
  const T be = (T)w.st[0].beta;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    p[i] = first ? z[i] : z[i] + be * p[i];
}

// x += alpha p; r -= alpha q; rr and the convergence test
template <typename T>
__global__ void __launch_bounds__(kKB) k_apcg_update(int nc, const T* p, const T* q, T* x, T* r, KWork w) {
  pdl_chain();
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

// ------------------------------------------------------------ host drivers
template <typename T>
struct AmgRun {
  difvm_mesh* m;
  const AmgHier* H;
  Topo t;
  Mat<T> A;
  char* ws;
  AmgLayout Ly;
  int G;
  int MW;
  // batched solves: the V-cycle's early exit reads this flag (1 once every case
  // has converged) and level 0 ends with a plain sweep (the per-case r.z follows)
  const int* seg_done = nullptr;
  // levels tail_from .. nlev-1 run in one cooperative launch of tail_grid
  // blocks (tail_from == 0: none)
  int tail_from = 0;
  int tail_grid = 0;
  T* vec(int k) const { return (T*)(ws + Ly.vec[k]); }
  T* at(size_t off) const { return (T*)(ws + off); }
};

// lanes per row of a level's sweeps: one on level 0 (the mesh's ELL); on a
// coarser level (never one lane: lev_row<T, 1> reads the mesh's ELL) two for
// large levels, 4-8 for small levels, whose sweeps are latency-bound chains of
// dependent loads (measured on the 1.6M-cell Kuhn mesh: 2 lanes on its
// 327k-row level 1 beat 4 and 8 by 2-7% of the step)
static int amg_tpr(const AmgLev& L, int l) {
  if (l == 0) return 1;
  if (L.n >= kAmgBigLevel) return 2;
  return L.nslots > 8 * L.n ? 8 : 4;
}

// Algorithmic bytes of the V-cycle kernels on level L (n rows, nf faces; next
// level n1 rows), element size v: the level's symmetric matrix is its faces'
// (owner, neighbour, coefficient) plus the diagonal; every vector a kernel
// reads or writes counts once.
static uint64_t lev_mat_bytes(const AmgLev& L, uint64_t v) { return (uint64_t)L.nf * (8 + v); }
static uint64_t lev_pre_bytes(const AmgLev& L, uint64_t v) { return lev_mat_bytes(L, v) + (uint64_t)L.n * 4 * v; }
static uint64_t lev_resid_bytes(const AmgLev& L, uint64_t v) { return lev_mat_bytes(L, v) + (uint64_t)L.n * 4 * v; }
static uint64_t lev_restrict_bytes(const AmgLev& L, int n1, uint64_t v) {
  return (uint64_t)L.n * (4 + v) + (uint64_t)n1 * 3 * v;   // children in; rD1 in, rc and sc out
}
static uint64_t lev_post1_bytes(const AmgLev& L, int n1, uint64_t v) {
  return lev_mat_bytes(L, v) + (uint64_t)L.n * (5 * v + 4) + (uint64_t)n1 * v;
}
static uint64_t lev_post2_bytes(const AmgLev& L, uint64_t v) { return lev_mat_bytes(L, v) + (uint64_t)L.n * 5 * v; }
// the correction in place: agg and y in, y out, the n1 coarse values once
static uint64_t lev_prol_bytes(const AmgLev& L, int n1, uint64_t v) {
  return (uint64_t)L.n * (4 + 2 * v) + (uint64_t)n1 * v;
}

// default launch shapes: lanes per row by amg_tpr; a restriction into a level
// of at least kAmgBigLevel/4 rows one thread per aggregate (four children in
// flight), into a smaller one eight lanes per aggregate
void amg_default_lanes(AmgHier* H) {
  H->tpr.assign(H->nlev, 1);
  H->rl.assign(H->nlev, 8);
  for (int l = 0; l < H->nlev; ++l) {
    H->tpr[l] = amg_tpr(H->lev[l], l);
    if (l + 1 < H->nlev) H->rl[l] = H->lev[l + 1].n >= kAmgBigLevel / 4 ? 1 : 8;
  }
}

// coarse operators of every level from the level-0 matrix (D, L symmetric)
template <typename T>
static difvm_status amg_setup(const AmgRun<T>& R, const T* D0, const T* L0, cudaStream_t st) {
  const AmgHier* H = R.H;
  const uint64_t v = sizeof(T);
  k_amg_rd<T><<<blocks_for(R.m->nc, kAB), kAB, 0, st>>>(R.m->nc, D0, R.at(R.Ly.rD[0]));
  DIFVM_TRY(check_launch("amg_rd"));
  count_bytes(2 * (uint64_t)R.m->nc * v);
  const T* D = D0;
  const T* Lv = L0;
  for (int l = 0; l + 1 < H->nlev; ++l) {
    const AmgLev& L = H->lev[l];
    const AmgLev& L1 = H->lev[l + 1];
    T *D1 = R.at(R.Ly.D[l + 1]), *rD1 = R.at(R.Ly.rD[l + 1]), *Lv1 = R.at(R.Ly.L[l + 1]);
    k_amg_diag<T><<<blocks_for(L1.n, kAB), kAB, 0, st>>>(L1.n, L, D, Lv, D1, rD1);
    // diagonal: the level's D, L and aggregate map in, D1 and 1/D1 out; faces: L in
    // with its map, L1 out; entries: L1 into the next level's ELL slots
    count_bytes((uint64_t)L.n * (v + 4) + (uint64_t)L.nf * (v + 4) + 2 * (uint64_t)L1.n * v);
    if (L1.nf > 0) count_bytes((uint64_t)L.nf * (v + 4) + (uint64_t)L1.nf * v +
                               (uint64_t)L1.nslots * (4 + v) + (uint64_t)L1.nf * v);
    if (L1.nf > 0) {
      k_amg_faces<T><<<blocks_for(L1.nf, kAB), kAB, 0, st>>>(L1.nf, L, Lv, Lv1);
      k_amg_entries<T><<<blocks_for(L1.nslots, kAB), kAB, 0, st>>>(L1.nslots, L1.eface, Lv1,
                                                                 R.at(R.Ly.E[l + 1]));
    }
    DIFVM_TRY(check_launch("amg_coarse_ops"));
    D = D1;
    Lv = Lv1;
  }
  const AmgLev& Lc = H->lev[H->nlev - 1];
  if (Lc.n > kAmgCoarsest) return set_error(DIFVM_EINVAL, "AMG: coarsest level has %d cells", Lc.n);
  k_amg_dense_inv<T><<<1, 512, 0, st>>>(Lc, D, Lv, (float*)(R.ws + R.Ly.inv));
  DIFVM_TRY(check_launch("amg_dense_inv"));
  count_bytes((uint64_t)Lc.n * Lc.n * 4 + (uint64_t)Lc.n * v + (uint64_t)Lc.nf * (8 + v));
  return DIFVM_OK;
}

// Levels below m->amg_tail_rows rows (and the coarsest solve) run in the fused
// kernel, with at most m->amg_tail_bps blocks per SM (default 2, at most its
// occupancy).  Off by default: on the 1.6M-cell Kuhn cavity the per-level
// kernels, chained by programmatic dependent launch, take 15.6 ms per PISO
// step against 16.0 ms with levels 3-6 fused and 16.5 ms with levels 2-6 (each
// phase has a fraction of the threads the per-level kernels keep resident, and
// the coarse phases are bound by the latency of their dependent loads).
static void amg_tail_plan(const difvm_mesh* m, const AmgHier* H, int elt, int& from, int& grid) {
  from = 0;
  grid = 0;
  const int mrows = m->amg_tail_rows >= 0 ? m->amg_tail_rows : 0;
  const int mbps = m->amg_tail_bps > 0 ? m->amg_tail_bps : 2;
  if (H->nlev < 2 || mrows <= 0) return;
  for (int l = 1; l < H->nlev; ++l)
    if (H->lev[l].n < mrows) {
      from = l;
      break;
    }
  if (from == 0) return;
  int bps = 0;
  const cudaError_t e = elt == 8
      ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_amg_tail<double>, kTB, 0)
      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_amg_tail<float>, kTB, 0);
  if (e != cudaSuccess || bps < 1) {
    from = 0;   // cannot be co-resident: keep the per-level kernels
    return;
  }
  grid = std::min(bps, mbps) * m->num_sms;
}

template <typename T>
static void amg_tail_launch(const AmgRun<T>& R, const int* done, KState* st, int nst, int* all_done,
                            cudaStream_t s) {
  TailArgs<T> a;
  a.lev = (const TailLev<T>*)(R.ws + R.Ly.tail);
  a.nlev = R.H->nlev - R.tail_from;
  a.Ainv = (const float*)(R.ws + R.Ly.inv);
  a.done = done;
  a.bar = (unsigned*)(R.ws + R.Ly.bar);
  a.st = st;
  a.nst = nst;
  a.all_done = all_done;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(R.tail_grid);
  cfg.blockDim = dim3(kTB);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;   // every block resident: the barriers complete
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_amg_tail<T>, a);   // an error is left for check_error
  count_launch();
}

template <typename T, int TPR>
static void amg_sweeps(const AmgRun<T>& R, const AmgLev& L, const AmgLev& L1, const T* D, const T* rD,
                       const T* Lv, const T* r, const T* sr, T* y, T* u, T* rc, const T* rD1, T* sc, T* xc,
                       T* out, const KWork& w, int first, int down, int rl, cudaStream_t s) {
  const int* done = R.seg_done ? R.seg_done : &w.st[0].done;
  const unsigned B = blocks_for((int64_t)L.n * TPR, kAB);
  const uint64_t v = sizeof(T);
  if (down) {
    count_bytes(lev_pre_bytes(L, v) + lev_resid_bytes(L, v) + lev_restrict_bytes(L, L1.n, v));
    if (sr)
      launch_pdl(k_amg_pre<T, TPR, true>, B, kAB, s, L, R.A, D, rD, Lv, r, sr, y, done);
    else
      launch_pdl(k_amg_pre<T, TPR, false>, B, kAB, s, L, R.A, D, rD, Lv, r, sr, y, done);
    if (TPR == 1) {
      prof_bytes(DIFVM_PROF_AMG_RESID, lev_resid_bytes(L, v));
      prof_before(DIFVM_PROF_AMG_RESID, s);
    }
    const bool co = L.n <= kAmgChildOrderRows;
    if (co)
      launch_pdl(k_amg_resid<T, TPR, true>, B, kAB, s, L, R.A, D, Lv, r, y, u, done);
    else
      launch_pdl(k_amg_resid<T, TPR, false>, B, kAB, s, L, R.A, D, Lv, r, y, u, done);
    if (TPR == 1) prof_after(DIFVM_PROF_AMG_RESID, s);
    const unsigned B1 = blocks_for(L1.n, kAB), B8 = blocks_for((int64_t)L1.n * 8, kAB);
    if (rl == 1 && co) launch_pdl(k_amg_restrict<T, 1, true>, B1, kAB, s, L1.n, L, u, rc, rD1, sc, done);
    else if (rl == 1) launch_pdl(k_amg_restrict<T, 1, false>, B1, kAB, s, L1.n, L, u, rc, rD1, sc, done);
    else if (co) launch_pdl(k_amg_restrict<T, 8, true>, B8, kAB, s, L1.n, L, u, rc, rD1, sc, done);
    else launch_pdl(k_amg_restrict<T, 8, false>, B8, kAB, s, L1.n, L, u, rc, rD1, sc, done);
    count_launch(); count_launch(); count_launch();
    return;
  }
  // a large level takes the correction in a kernel of its own (one gather per
  // row) and then sweeps with one gather per column (64^3 cavity: 15.35 -> 14.97
  // ms per step with the mesh level and the 327k-row level so); small levels,
  // whose kernels are bound by launch and latency, form it on the fly
  const bool sep = L.n >= kAmgBigLevel;
  const uint64_t b1 = sep ? lev_prol_bytes(L, L1.n, v) + lev_post2_bytes(L, v) : lev_post1_bytes(L, L1.n, v);
  count_bytes(b1 + lev_post2_bytes(L, v));
  if (sep) {
    launch_pdl(k_amg_prol<T>, blocks_for(L.n, kAB), kAB, s, L, (const T*)xc, y, done);
    count_launch();
  }
  if (TPR == 8) {
    prof_bytes(DIFVM_PROF_AMG_POST1C, b1);
    prof_before(DIFVM_PROF_AMG_POST1C, s);
  }
  if (sep)
    launch_pdl(k_amg_post1<T, TPR, true>, B, kAB, s, L, R.A, D, rD, Lv, r, y, xc, u, done);
  else
    launch_pdl(k_amg_post1<T, TPR, false>, B, kAB, s, L, R.A, D, rD, Lv, r, y, xc, u, done);
  if (TPR == 8) prof_after(DIFVM_PROF_AMG_POST1C, s);
  if (TPR == 1 && !R.seg_done)
    launch_pdl(k_amg_post2_dot<T>, R.G, kKB, s, L, R.A, rD, r, u, out, w, first);
  else
    launch_pdl(k_amg_post2<T, TPR>, B, kAB, s, L, R.A, D, rD, Lv, r, u, out, done);
  count_launch(); count_launch();
}

// z = V-cycle(r) on level l; level 0 ends with the r.z reduction of the CG
template <typename T>
static void amg_vcycle(const AmgRun<T>& R, int l, const T* r, T* out, const KWork& w, int first,
                       cudaStream_t s) {
  const AmgHier* H = R.H;
  const AmgLev& L = H->lev[l];
  const int* done = R.seg_done ? R.seg_done : &w.st[0].done;
  if (R.tail_from > 0 && l == R.tail_from) {
    const uint64_t v = sizeof(T);
    for (int k = l; k + 1 < H->nlev; ++k) {
      const AmgLev& Lk = H->lev[k];
      const int n1 = H->lev[k + 1].n;
      count_bytes(lev_pre_bytes(Lk, v) + lev_resid_bytes(Lk, v) + lev_restrict_bytes(Lk, n1, v) +
                  lev_post1_bytes(Lk, n1, v) + lev_post2_bytes(Lk, v));
    }
    const int nco = H->lev[H->nlev - 1].n;
    count_bytes((uint64_t)nco * nco * 4 + 2 * (uint64_t)nco * v);
    KState* st = (KState*)(R.ws + R.Ly.st);
    amg_tail_launch(R, done, R.seg_done ? st : w.st, R.seg_done ? R.m->ncases : 1,
                    R.seg_done ? const_cast<int*>(R.seg_done) : nullptr, s);
    return;
  }
  const bool fine = l == 0;
  const T* D = fine ? R.A.D : R.at(R.Ly.D[l]);
  const T* rD = R.at(R.Ly.rD[l]);
  const T* Lv = fine ? nullptr : R.at(R.Ly.E[l]);   // row-entry values of a coarse level
  if (l == H->nlev - 1) {
    count_bytes((uint64_t)L.n * L.n * 4 + 2 * (uint64_t)L.n * sizeof(T));
    // one warp per row, spread over blocks so that every row is one round of loads
    launch_pdl(k_amg_coarse<T>, std::max(1, (L.n + kAmgCoarseTB / 32 - 1) / (kAmgCoarseTB / 32)), kAmgCoarseTB, s,
               L.n, (const float*)(R.ws + R.Ly.inv), r, out, done);
    count_launch();
    if (l == 0 && !R.seg_done) {   // a single level: the CG's r.z reduction runs on its own
      k_apcg_rz<T><<<R.G, kKB, 0, s>>>(L.n, r, out, w, first);
      count_launch();
    }
    return;
  }
  T *y = R.at(R.Ly.a[l]), *u = R.at(R.Ly.b[l]);
  const AmgLev& L1 = H->lev[l + 1];
  T* rc = R.at(R.Ly.r[l + 1]);
  T* sc = R.at(R.Ly.s[l + 1]);
  const T* rD1 = R.at(R.Ly.rD[l + 1]);
  const T* sr = fine ? nullptr : R.at(R.Ly.s[l]);   // formed by the restriction into this level
  T* xc = R.at(R.Ly.a[l + 1]);   // written by the next level's last sweep
  const int tpr = H->tpr[l], rl = H->rl[l];
#define DIFVM_SWEEPS(TPRc) \
  amg_sweeps<T, TPRc>(R, L, L1, D, rD, Lv, r, sr, y, u, rc, rD1, sc, xc, out, w, first, down, rl, s)
  for (int down = 1; down >= 0; --down) {
    if (tpr == 1) DIFVM_SWEEPS(1);
    else if (tpr == 2) DIFVM_SWEEPS(2);
    else if (tpr == 4) DIFVM_SWEEPS(4);
    else DIFVM_SWEEPS(8);
    if (down) amg_vcycle(R, l + 1, rc, xc, w, first, s);
  }
#undef DIFVM_SWEEPS
}

// one AMG-preconditioned CG solve of A x = b (x is the initial guess unless
// zero_x); state in w.st[0]; `gate` closes the solve at once when set
template <typename T, int MW>
static difvm_status amg_cg(const AmgRun<T>& R, const T* b, T* x, const KWork& w, const int* gate,
                           int zero_x, int chunk, cudaStream_t st) {
  const int nc = R.m->nc, G = R.G;
  T *r = R.vec(0), *p = R.vec(1), *q = R.vec(2), *z = R.vec(3);
  k_apcg_init<T, MW><<<G, kKB, 0, st>>>(R.t, R.A, b, x, r, w, gate, zero_x);
  DIFVM_TRY(check_launch("apcg_init"));
  k_apcg_zero<T><<<G, kKB, 0, st>>>(nc, x, w);
  DIFVM_TRY(check_launch("apcg_zero"));
  amg_vcycle(R, 0, r, z, w, 1, st);
  k_apcg_p<T><<<G, kKB, 0, st>>>(nc, z, p, w, 1);
  DIFVM_TRY(check_launch("apcg_p"));
  const uint64_t v = sizeof(T), n64 = (uint64_t)nc;
  const uint64_t cg_bytes = lev_mat_bytes(R.H->lev[0], v) + 3 * n64 * v + 6 * n64 * v + 3 * n64 * v;
  auto iter = [&](cudaStream_t s) {
    count_bytes(cg_bytes);   // q = A p; x, r update; p update
    prof_before(DIFVM_PROF_PCG_SPMV, s);
    k_pcg_spmv<T, 1, MW><<<G, kKB, 0, s>>>(R.t, R.A, p, q, w);
    prof_after(DIFVM_PROF_PCG_SPMV, s);
    launch_pdl(k_apcg_update<T>, G, kKB, s, nc, p, q, x, r, w);
    amg_vcycle(R, 0, r, z, w, 0, s);
    launch_pdl(k_apcg_p<T>, G, kKB, s, nc, z, p, w, 0);
    count_launch(); count_launch(); count_launch();
  };
  int* counter = reinterpret_cast<int*>(w.ticket) + 1;
  if (stream_capturing(st)) {
    DIFVM_CUDA(cudaMemsetAsync(counter, 0, sizeof(int), st));
    WhileLoop Lw;
    DIFVM_TRY(while_open(st, Lw));
    iter(Lw.side);
    k_loop_cond<<<1, 32, 0, Lw.side>>>(done_flags(w.st), kStateInts, 1, counter, w.maxit + 2, Lw.h);
    difvm_status e = check_launch("loop_cond");
    DIFVM_TRY(while_close(Lw));
    return e;
  }
  KState hs;
  for (int it = 0; it < w.maxit + chunk; it += chunk) {
    for (int k = 0; k < chunk; ++k) iter(st);
    DIFVM_TRY(check_error("apcg_iter"));
    DIFVM_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
    DIFVM_CUDA(cudaStreamSynchronize(st));
    if (hs.done) break;
  }
  return DIFVM_OK;
}

__global__ void k_amg_info(const KState* st, difvm_solve_info* info, int refinements, int iters) {
  if (threadIdx.x != 0) return;
  difvm_solve_info o;
  o.iters = iters >= 0 ? iters : st->iters;
  o.refinements = refinements;
  o.status = st->status;
  o.pad = 0;
  o.res0 = st->res0;
  o.res = sqrt(st->rr);
  o.bnorm = sqrt(st->bb);
  *info = o;
}

// the fused kernel's level descriptors (pointers into this workspace and the
// current launch shapes), written at every solve so that a change of the
// mesh's configuration or launch shapes between solves is always seen
template <typename T>
static difvm_status amg_tail_descs(const AmgRun<T>& R, cudaStream_t st) {
  const AmgHier* H = R.H;
  if (R.tail_from > 0) {
    TailLevs<T> d;
    const int nl = H->nlev - R.tail_from;
    for (int k = 0; k < nl; ++k) {
      const int l = R.tail_from + k;
      const AmgLev& L = H->lev[l];
      TailLev<T>& t = d.lev[k];
      t.L = L;
      t.D = R.at(R.Ly.D[l]);
      t.rD = R.at(R.Ly.rD[l]);
      t.Lv = R.at(R.Ly.E[l]);
      t.r = R.at(R.Ly.r[l]);
      t.y = R.at(R.Ly.a[l]);
      t.u = R.at(R.Ly.b[l]);
      t.tpr = H->tpr[l];
      t.rl = H->rl[l];
    }
    k_amg_tail_desc<T><<<1, 32, 0, st>>>(d, nl, (TailLev<T>*)(R.ws + R.Ly.tail));
    DIFVM_TRY(check_launch("amg_tail_desc"));
  }
  return DIFVM_OK;
}


// reuse: the ELL values and multigrid operators already in the workspace belong to
// this same matrix (DIFVM_PRECOND_AMG_REUSE); only the views are set up
template <typename T>
static difvm_status amg_prepare(difvm_mesh* m, const T* D, const T* Lo, void* ws, size_t wsbytes,
                                AmgRun<T>& R, cudaStream_t st, bool reuse = false) {
  AmgHier* H = nullptr;
  DIFVM_TRY(amg_hier(m, &H));
  R.m = m;
  R.H = H;
  R.t = m->topo();
  R.ws = (char*)ws;
  R.Ly = amg_layout(m, H, sizeof(T));
  if (!ws || wsbytes < R.Ly.total)
    return set_error(DIFVM_EINVAL, "workspace of %zu bytes < %zu needed (AMG)", wsbytes, R.Ly.total);
  R.G = amg_grid(m);
  amg_tail_plan(m, H, (int)sizeof(T), R.tail_from, R.tail_grid);
  if (R.tail_from > 0) DIFVM_CUDA(cudaMemsetAsync(R.ws + R.Ly.bar, 0, sizeof(unsigned), st));
  DIFVM_TRY(amg_tail_descs(R, st));
  T* val = R.at(R.Ly.val);
  if (reuse) {
    R.A = Mat<T>{D, m->ell(), val};
    return DIFVM_OK;
  }
  if (m->ell_nslots > 0) {
    k_ell_fill<T><<<blocks_for(m->ell_nslots, 256), 256, 0, st>>>((int)m->ell_nslots, m->ell_map, Lo, Lo, val);
    DIFVM_TRY(check_launch("ell_fill"));
    count_bytes((uint64_t)m->ni * sizeof(T) + 2 * (uint64_t)m->ni * (4 + sizeof(T)));
  }
  R.A = Mat<T>{D, m->ell(), val};
  return amg_setup(R, D, Lo, st);
}

template <typename T>
static KWork amg_work_t(const AmgRun<T>& R, int k, int maxit, double tol_rel, double tol_abs) {
  KWork w;
  w.st = (KState*)(R.ws + R.Ly.st) + k;
  w.part = (double*)(R.ws + R.Ly.part);
  w.ticket = (unsigned*)(R.ws + R.Ly.ticket);
  w.maxit = maxit;
  w.tol_rel = tol_rel;
  w.tol_abs = tol_abs;
  return w;
}

// Autotuning of the V-cycle's launch shapes, once per hierarchy: whole FP32
// V-cycles, launched exactly as the solvers launch them (programmatic
// dependent launch), are timed on a temporary workspace whose operators and
// vectors are zero (the timing of these gathers does not depend on the
// values).  Level by level below the mesh level, the lanes per row of the
// level's sweeps (2, 4, 8) and then the lanes per aggregate of its restriction
// (1, 8) are varied with the other levels fixed, and a shape replaces the
// current one only if the V-cycle is at least 2% faster.  The workspace is
// freed afterwards; on any CUDA error the defaults stay.  Results go to the
// mesh's tuning record: key 5 << 8 | level << 4 -> lanes per row,
// 6 << 8 | level << 4 -> restriction lanes.
void amg_tune(difvm_mesh* m, AmgHier* H) {
  amg_default_lanes(H);
  const int nl = H->nlev;
  if (nl < 3) return;
  AmgRun<float> R;
  R.m = m;
  R.H = H;
  R.t = m->topo();
  R.Ly = amg_layout(m, H, 4);
  R.G = amg_grid(m);
  const size_t bytes = R.Ly.total + ((size_t)m->nc * 4 + 255) / 256 * 256;
  char* ws = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc((void**)&ws, bytes) != cudaSuccess || cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (ws) cudaFree(ws);
    if (s) cudaStreamDestroy(s);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    return;
  }
  cudaMemsetAsync(ws, 0, bytes, s);
  R.ws = ws;
  R.A = Mat<float>{(const float*)(ws + R.Ly.total), m->ell(), R.at(R.Ly.val)};
  const KWork w = amg_work_t(R, 0, 1000, 0.0, 0.0);   // zeroed state: nothing converged
  count_bytes_pause(true);
  auto vcycles = [&]() -> float {
    constexpr int kWarm = 2, kReps = 6;
    for (int k = 0; k < kWarm; ++k) amg_vcycle(R, 0, R.vec(0), R.vec(3), w, 0, s);
    cudaEventRecord(e0, s);
    for (int k = 0; k < kReps; ++k) amg_vcycle(R, 0, R.vec(0), R.vec(3), w, 0, s);
    cudaEventRecord(e1, s);
    float ms = -1.f;
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) ms = -1.f;
    return ms;
  };
  bool ok = true;
  float cur = vcycles();
  ok = cur > 0.f;
  auto try_shapes = [&](std::vector<int>& field, int l, std::initializer_list<int> cands) {
    const int keep = field[l];
    int best = keep;
    float best_t = cur;
    for (int c : cands) {
      if (c == keep || !ok) continue;
      field[l] = c;
      const float t = vcycles();
      if (t < 0.f) { ok = false; break; }
      if (t < 0.98f * best_t) { best_t = t; best = c; }
    }
    field[l] = best;
    cur = best_t;
  };
  for (int l = 1; l + 1 < nl && ok; ++l) {
    try_shapes(H->tpr, l, {2, 4, 8});
    try_shapes(H->rl, l, {1, 8});
  }
  count_bytes_pause(false);
  cudaStreamSynchronize(s);
  ok = ok && cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(s);
  cudaFree(ws);
  cudaGetLastError();
  if (!ok) {
    amg_default_lanes(H);
    return;
  }
  auto keep = [&](uint32_t key, int val) {
    for (auto& kv : m->tuned)
      if (kv.first == key) { kv.second = val; return; }
    m->tuned.emplace_back(key, val);
  };
  for (int l = 1; l + 1 < nl; ++l) {
    keep((uint32_t)(5 << 8 | l << 4), H->tpr[l]);
    keep((uint32_t)(6 << 8 | l << 4), H->rl[l]);
  }
}

// Build the ELL values and multigrid operators of the matrix (D, Lo) in the
// workspace, so that a following AMG_REUSE solve with this workspace starts at
// once (the PISO step builds them beside its momentum solve).  elt = 4: FP32
// operators (FP32 solves and the mixed-precision solve), 8: FP64.
difvm_status amg_prebuild(difvm_mesh* m, size_t elt, const void* D, const void* Lo, void* ws, size_t wsbytes,
                          cudaStream_t st) {
  if (elt == 8) {
    AmgRun<double> R;
    return amg_prepare<double>(m, (const double*)D, (const double*)Lo, ws, wsbytes, R, st, false);
  }
  AmgRun<float> R;
  return amg_prepare<float>(m, (const float*)D, (const float*)Lo, ws, wsbytes, R, st, false);
}

template <typename T, int MW>
static difvm_status amg_solve_mw(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo,
                                 const T* b, T* x, void* ws, size_t wsbytes, difvm_solve_info* info,
                                 cudaStream_t st) {
  AmgRun<T> R;
  DIFVM_TRY(amg_prepare<T>(m, D, Lo, ws, wsbytes, R, st, o->precond == DIFVM_PRECOND_AMG_REUSE));
  KWork w = amg_work_t(R, 0, o->max_iter > 0 ? o->max_iter : 1000, o->tol_rel, o->tol_abs);
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned), st));
  const int chunk = o->check_every > 0 ? o->check_every : 8;
  DIFVM_TRY((amg_cg<T, MW>(R, b, x, w, nullptr, 0, chunk, st)));
  if (info) {
    k_amg_info<<<1, 32, 0, st>>>(w.st, info, 0, -1);
    DIFVM_TRY(check_launch("amg_info"));
  }
  if (stream_capturing(st)) return DIFVM_OK;
  KState hs;
  DIFVM_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  return (difvm_status)hs.status;
}

// ------------------------------------------------- batched (segmented) CG
// The multigrid-preconditioned CG on a disjoint union of cases.  Every case keeps
// its own CG scalars, convergence flag and iteration count, with the per-case
// reductions of the segmented Krylov solvers (seg_sum).  The hierarchy is built
// on the union: an aggregate only joins cells linked by a face, so it never
// spans two cases, every coarse operator is block diagonal by case and one
// V-cycle over the union applies each case's own V-cycle.  flag[0] counts the
// converged cases and flag[1] turns 1 once all have converged: the V-cycle
// kernels then return at once.
__device__ __forceinline__ void sg_case_done(int* flag, int ncases) {
  if (atomicAdd(flag, 1) + 1 == ncases) atomicExch(flag + 1, 1);
}

// r = b - A x; bb, rr per case; convergence at the start
template <typename T, int MW>
__global__ void __launch_bounds__(kKB) k_sgapcg_init(Topo t, Mat<T> A, const T* b, const T* x, T* r,
                                                      SWork w, int* flag, int ncases) {
  const SegBlock B = seg_block(w);
  DotAcc<T> bb, rr;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    T ax[1];
    spmv_row<T, 1, MW>(t, A, i, x, ax, 1u);
    const T bi = b[i], ri = bi - ax[0];
    r[i] = ri;
    bb.add(bi, bi);
    rr.add(ri, ri);
  }
  double v[2] = {bb.get(), rr.get()}, tot[2];
  if (!seg_sum<2>(w, B.k, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[B.k];
  s.bb = tot[0];
  s.rr = tot[1];
  s.res0 = sqrt(s.rr);
  s.tol2 = fmax(w.tol_rel * w.tol_rel * s.bb, w.tol_abs * w.tol_abs);
  s.iters = 0;
  s.status = DIFVM_OK;
  s.zero_rhs = s.bb == 0.0;
  s.done = s.zero_rhs || s.rr <= s.tol2;
  if (!isfinite(s.rr)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
  if (s.done) sg_case_done(flag, ncases);
}

// a case with b = 0 gets x = 0
template <typename T>
__global__ void k_sgapcg_zero(T* x, SWork w) {
  const SegBlock B = seg_block(w);
  if (!w.st[B.k].zero_rhs) return;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) x[i] = T(0);
}

// r.z of each active case and its beta (first: beta = 0)
template <typename T>
__global__ void __launch_bounds__(kKB) k_sgapcg_rz(const T* r, const T* z, SWork w, int first) {
  pdl_chain();
  const SegBlock B = seg_block(w);
  if (w.st[B.k].done) return;
  DotAcc<T> rz;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) rz.add(r[i], z[i]);
  double v[1] = {rz.get()}, tot[1];
  if (!seg_sum<1>(w, B.k, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[B.k];
  s.beta = first ? 0.0 : tot[0] / s.rz;
  s.rz = tot[0];
}

// p = z + beta p in each active case (first: p = z)
template <typename T>
__global__ void __launch_bounds__(kKB) k_sgapcg_p(const T* z, T* p, SWork w, int first) {
  pdl_chain();
  const SegBlock B = seg_block(w);
  if (w.st[B.k].done) return;
  const T be = (T)w.st[B.k].beta;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) p[i] = first ? z[i] : z[i] + be * p[i];
}

// q = A p in each active case; alpha = rz / (p.q)
template <typename T, int MW>
__global__ void __launch_bounds__(kKB) k_sgapcg_spmv(Topo t, Mat<T> A, const T* p, T* q, SWork w) {
  pdl_chain();
  const SegBlock B = seg_block(w);
  if (w.st[B.k].done) return;
  DotAcc<T> pq;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    T y[1];
    spmv_row<T, 1, MW>(t, A, i, p, y, 1u);
    q[i] = y[0];
    pq.add(p[i], y[0]);
  }
  double v[1] = {pq.get()}, tot[1];
  if (!seg_sum<1>(w, B.k, v, tot) || threadIdx.x != 0) return;
  w.st[B.k].alpha = w.st[B.k].rz / tot[0];
}

// x += alpha p; r -= alpha q; rr and the convergence test of each active case
template <typename T>
__global__ void __launch_bounds__(kKB) k_sgapcg_update(const T* p, const T* q, T* x, T* r, SWork w,
                                                        int* flag, int ncases) {
  pdl_chain();
  const SegBlock B = seg_block(w);
  if (w.st[B.k].done) return;
  const T al = (T)w.st[B.k].alpha;
  DotAcc<T> rr;
  for (int i = B.r0 + threadIdx.x; i < B.r1; i += blockDim.x) {
    x[i] += al * p[i];
    const T ri = r[i] - al * q[i];
    r[i] = ri;
    rr.add(ri, ri);
  }
  double v[1] = {rr.get()}, tot[1];
  if (!seg_sum<1>(w, B.k, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[B.k];
  s.iters += 1;
  s.rr = tot[0];
  if (!isfinite(s.rr) || !isfinite(s.alpha)) { s.done = 1; s.status = DIFVM_ENONFINITE; }
  else if (s.rr <= s.tol2) s.done = 1;
  else if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; }
  if (s.done) sg_case_done(flag, ncases);
}

__global__ void k_sgapcg_info(int n, const KState* st, difvm_solve_info* info) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const KState& s = st[c];
  difvm_solve_info o;
  o.iters = s.iters;
  o.refinements = 0;
  o.status = s.status;
  o.pad = 0;
  o.res0 = s.res0;
  o.res = sqrt(s.rr);
  o.bnorm = sqrt(s.bb);
  info[c] = o;
}

template <typename T, int MW>
static difvm_status amg_solve_seg(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo,
                                  const T* b, T* x, void* ws, size_t wsbytes, difvm_solve_info* info,
                                  cudaStream_t st) {
  AmgRun<T> R;
  DIFVM_TRY(amg_prepare<T>(m, D, Lo, ws, wsbytes, R, st, o->precond == DIFVM_PRECOND_AMG_REUSE));
  const int nk = m->ncases, G = m->seg_nblk;
  SWork w;
  w.st = (KState*)(R.ws + R.Ly.st);
  w.part = (double*)(R.ws + R.Ly.part);
  w.ticket = (unsigned*)(R.ws + R.Ly.ticket);
  w.bcase = m->seg_case;
  w.cb0 = m->seg_cb0;
  w.cs = m->seg_cs;
  w.maxit = o->max_iter > 0 ? o->max_iter : 1000;
  w.tol_rel = o->tol_rel;
  w.tol_abs = o->tol_abs;
  int* flag = (int*)(R.ws + R.Ly.flag);   // converged cases, all converged, loop counter, poll
  R.seg_done = flag + 1;
  KWork kw = amg_work_t(R, 0, w.maxit, w.tol_rel, w.tol_abs);   // (unused by a batched V-cycle)
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, sizeof(unsigned) * nk, st));
  DIFVM_CUDA(cudaMemsetAsync(flag, 0, 4 * sizeof(int), st));
  T *r = R.vec(0), *p = R.vec(1), *q = R.vec(2), *z = R.vec(3);
  k_sgapcg_init<T, MW><<<G, kKB, 0, st>>>(R.t, R.A, b, x, r, w, flag, nk);
  k_sgapcg_zero<T><<<G, kKB, 0, st>>>(x, w);
  DIFVM_TRY(check_launch("sgapcg_init"));
  amg_vcycle(R, 0, r, z, kw, 1, st);
  launch_pdl(k_sgapcg_rz<T>, G, kKB, st, (const T*)r, (const T*)z, w, 1);
  launch_pdl(k_sgapcg_p<T>, G, kKB, st, (const T*)z, p, w, 1);
  DIFVM_TRY(check_launch("sgapcg_first"));
  auto iter = [&](cudaStream_t s) {
    launch_pdl(k_sgapcg_spmv<T, MW>, G, kKB, s, R.t, R.A, (const T*)p, q, w);
    launch_pdl(k_sgapcg_update<T>, G, kKB, s, (const T*)p, (const T*)q, x, r, w, flag, nk);
    amg_vcycle(R, 0, r, z, kw, 0, s);
    launch_pdl(k_sgapcg_rz<T>, G, kKB, s, (const T*)r, (const T*)z, w, 0);
    launch_pdl(k_sgapcg_p<T>, G, kKB, s, (const T*)z, p, w, 0);
    for (int k = 0; k < 4; ++k) count_launch();
  };
  if (stream_capturing(st)) {
    WhileLoop Lw;
    DIFVM_TRY(while_open(st, Lw));
    iter(Lw.side);
    // continue while flag[1] == 0, at most maxit + 2 passes
    k_loop_cond<<<1, 32, 0, Lw.side>>>(flag + 1, 0, 1, flag + 2, w.maxit + 2, Lw.h);
    DIFVM_TRY(check_launch("loop_cond"));
    DIFVM_TRY(while_close(Lw));
  } else {
    const int chunk = o->check_every > 0 ? o->check_every : 8;
    int all = 0;
    for (int it = 0; it < w.maxit && !all; it += chunk) {
      for (int k = 0; k < chunk; ++k) iter(st);
      DIFVM_TRY(check_error("sgapcg_iter"));
      DIFVM_CUDA(cudaMemcpyAsync(&all, flag + 1, sizeof(int), cudaMemcpyDeviceToHost, st));
      DIFVM_CUDA(cudaStreamSynchronize(st));
    }
  }
  if (info) {
    k_sgapcg_info<<<blocks_for(nk, 128), 128, 0, st>>>(nk, w.st, info);
    DIFVM_TRY(check_launch("sgapcg_info"));
  }
  if (stream_capturing(st)) return DIFVM_OK;   // outcome in info_dev
  std::vector<KState> hs(nk);
  DIFVM_CUDA(cudaMemcpyAsync(hs.data(), w.st, sizeof(KState) * nk, cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  int worst = DIFVM_OK;
  for (const KState& k : hs) worst = std::max(worst, k.status);
  return (difvm_status)worst;
}

template <typename T>
difvm_status amg_solve(difvm_mesh* m, const difvm_solve_opts* o, const T* D, const T* Lo, const T* b,
                       T* x, void* ws, size_t wsbytes, difvm_solve_info* info, cudaStream_t st) {
  if (m->seg) {
    if (m->ell_wmax <= 4) return amg_solve_seg<T, 4>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
    if (m->ell_wmax <= 8) return amg_solve_seg<T, 8>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
    return amg_solve_seg<T, 0>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
  }
  if (m->ell_wmax <= 4) return amg_solve_mw<T, 4>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
  if (m->ell_wmax <= 8) return amg_solve_mw<T, 8>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
  return amg_solve_mw<T, 0>(m, o, D, Lo, b, x, ws, wsbytes, info, st);
}
template difvm_status amg_solve<float>(difvm_mesh*, const difvm_solve_opts*, const float*, const float*,
                                       const float*, float*, void*, size_t, difvm_solve_info*, cudaStream_t);
template difvm_status amg_solve<double>(difvm_mesh*, const difvm_solve_opts*, const double*, const double*,
                                        const double*, double*, void*, size_t, difvm_solve_info*,
                                        cudaStream_t);

// ------------------------------------------------------ mixed precision
// CG with FP64 accuracy around the FP32 V-cycle.  The preconditioner's
// precision only affects the convergence rate, so the solve reaches FP64
// tolerances without refinement sweeps or restarts.  The CG vectors x, r, p, q
// are float-float pairs (hi, lo: about 48 significant bits) updated with
// error-free transformations (TwoSum: Knuth; TwoProduct by fma), so the B300's
// FP32 pipes carry what FP64 arithmetic would (its FP64 rate is ~1/64 of
// FP32); inner products are reduced in FP64.  The initial residual b - A x and
// the returned x are FP64; the FP32 coefficients are exact in either form.
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast_two_sum(float a, float b) {   // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = ff_two_sum(x.h, y.h);
  return ff_fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}
__device__ __forceinline__ FF ff_mul_f(FF x, float a) {            // x * a
  const float p = __fmul_rn(x.h, a);
  const float e = __fmaf_rn(x.h, a, -p);
  return ff_fast_two_sum(p, __fmaf_rn(x.l, a, e));
}
__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const float p = __fmul_rn(x.h, y.h);
  float e = __fmaf_rn(x.h, y.h, -p);
  e = __fmaf_rn(x.h, y.l, e);
  e = __fmaf_rn(x.l, y.h, e);
  return ff_fast_two_sum(p, e);
}
__device__ __forceinline__ FF ff_of(double d) {
  const float h = (float)d;
  return FF{h, (float)(d - (double)h)};
}
__device__ __forceinline__ double ff_dbl(FF x) { return (double)x.h + (double)x.l; }

// r = b - A x in FP64 (stored as pairs), x as pairs; bb, rr
template <int MW>
__global__ void __launch_bounds__(kKB) k_fcg_init(Topo t, Mat<float> A, const double* b, const double* x,
                                                  float* xh, float* xl, float* rh, float* rl, KWork w) {
  const int nc = t.nc;
  double bb = 0.0, rr = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    double y = (double)A.D[i] * x[i];
    if (MW == 4 && A.E.W == 4) {
      const int4 j4 = ell_cols4(A.E, i);
      const float4 a4 = __ldg(reinterpret_cast<const float4*>(A.val) + i);
      y = fma((double)a4.x, x[j4.x], y);
      y = fma((double)a4.y, x[j4.y], y);
      y = fma((double)a4.z, x[j4.z], y);
      y = fma((double)a4.w, x[j4.w], y);
    } else {
      int base, step, wd;
      ell_row(A.E, i, base, step, wd);
      for (int k = 0; k < wd; ++k) y = fma((double)A.val[base + step * k], x[A.E.col[base + step * k]], y);
    }
    const double ri = b[i] - y;
    const FF rf = ff_of(ri), xf = ff_of(x[i]);
    rh[i] = rf.h;
    rl[i] = rf.l;
    xh[i] = xf.h;
    xl[i] = xf.l;
    bb = fma(b[i], b[i], bb);
    rr = fma(ri, ri, rr);
  }
  double v[2] = {bb, rr}, tot[2];
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

// q = A p (pairs; FP32 coefficients); alpha = rz / (p.q)
template <int MW>
__global__ void __launch_bounds__(kKB) k_fcg_spmv(Topo t, Mat<float> A, const float* ph, const float* pl,
                                                  float* qh, float* ql, KWork w) {
  pdl_chain();
  if (w.st[0].done) return;
  const int nc = t.nc;
  FF pq{0.f, 0.f};
  auto pv = [&](int j) { return FF{__ldg(ph + j), __ldg(pl + j)}; };
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const FF pi = pv(i);
    FF y = ff_mul_f(pi, __ldg(A.D + i));
    if (MW == 4 && A.E.W == 4) {
      const int4 j4 = ell_cols4(A.E, i);
      const float4 a4 = __ldg(reinterpret_cast<const float4*>(A.val) + i);
      const FF p0 = pv(j4.x), p1 = pv(j4.y), p2 = pv(j4.z), p3 = pv(j4.w);
      y = ff_add(y, ff_mul_f(p0, a4.x));
      y = ff_add(y, ff_mul_f(p1, a4.y));
      y = ff_add(y, ff_mul_f(p2, a4.z));
      y = ff_add(y, ff_mul_f(p3, a4.w));
    } else {
      int base, step, wd;
      ell_row(A.E, i, base, step, wd);
      for (int k = 0; k < wd; ++k)
        y = ff_add(y, ff_mul_f(pv(__ldg(A.E.col + base + step * k)), __ldg(A.val + base + step * k)));
    }
    qh[i] = y.h;
    ql[i] = y.l;
    pq = ff_add(pq, ff_mul(pi, y));
  }
  double v[1] = {ff_dbl(pq)}, tot[1];
  if (!grid_sum<1>(w, v, tot) || threadIdx.x != 0) return;
  w.st[0].alpha = w.st[0].rz / tot[0];
}

// x += alpha p; r -= alpha q (pairs); rr; convergence
__global__ void __launch_bounds__(kKB) k_fcg_update(int nc, const float* ph, const float* pl, const float* qh,
                                                    const float* ql, float* xh, float* xl, float* rh, float* rl,
                                                    KWork w) {
  pdl_chain();
  if (w.st[0].done) return;
  const FF al = ff_of(w.st[0].alpha), nal = ff_of(-w.st[0].alpha);
  FF rr{0.f, 0.f};
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const FF p{ph[i], pl[i]}, q{qh[i], ql[i]};
    const FF x = ff_add(FF{xh[i], xl[i]}, ff_mul(p, al));
    const FF r = ff_add(FF{rh[i], rl[i]}, ff_mul(q, nal));
    xh[i] = x.h;
    xl[i] = x.l;
    rh[i] = r.h;
    rl[i] = r.l;
    rr = ff_add(rr, ff_mul(r, r));
  }
  double v[1] = {ff_dbl(rr)}, tot[1];
  if (!grid_sum<1>(w, v, tot) || threadIdx.x != 0) return;
  KState& s = w.st[0];
  s.iters += 1;
  s.rr = tot[0];
  if (!isfinite(s.rr) || !isfinite(s.alpha)) { s.done = 1; s.status = DIFVM_ENONFINITE; return; }
  if (s.rr <= s.tol2) { s.done = 1; return; }
  if (s.iters >= w.maxit) { s.done = 1; s.status = DIFVM_ENOTCONV; }
}

// p = z + beta p (first: p = z)
__global__ void __launch_bounds__(kKB) k_fcg_p(int nc, const float* z, float* ph, float* pl, KWork w, int first) {
  pdl_chain();
  if (w.st[0].done) return;
  const FF be = ff_of(w.st[0].beta);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x) {
    const FF p = first ? FF{z[i], 0.f} : ff_add(ff_mul(FF{ph[i], pl[i]}, be), FF{z[i], 0.f});
    ph[i] = p.h;
    pl[i] = p.l;
  }
}

// x64 = xh + xl (0 for a zero right-hand side)
__global__ void k_fcg_final(int nc, const float* xh, const float* xl, double* x, KWork w) {
  const bool z = w.st[0].zero_rhs;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nc; i += gridDim.x * blockDim.x)
    x[i] = z ? 0.0 : (double)xh[i] + (double)xl[i];
}

template <int MW>
static difvm_status amg_mixed_mw(difvm_mesh* m, const difvm_solve_opts* o, const float* D, const float* Lo,
                                 const double* b64, double* x64, void* ws, size_t wsbytes,
                                 difvm_solve_info* info, cudaStream_t st) {
  AmgRun<float> R;
  DIFVM_TRY(amg_prepare<float>(m, D, Lo, ws, wsbytes, R, st, o->precond == DIFVM_PRECOND_AMG_REUSE));
  const size_t vb = up256a((size_t)m->nc * 4);
  if (R.Ly.total + 7 * vb > wsbytes)
    return set_error(DIFVM_EINVAL, "workspace of %zu bytes < %zu needed (AMG)", wsbytes, R.Ly.total + 7 * vb);
  float* base = (float*)(R.ws + R.Ly.total);
  float *xh = base, *xl = base + vb / 4, *rl = base + 2 * vb / 4, *ph = base + 3 * vb / 4;
  float *pl = base + 4 * vb / 4, *qh = base + 5 * vb / 4, *ql = base + 6 * vb / 4;
  float* rh = R.vec(0);    // the V-cycle's input
  float* z32 = R.vec(3);
  KWork w = amg_work_t(R, 0, o->max_iter > 0 ? o->max_iter : 1000, o->tol_rel, o->tol_abs);
  DIFVM_CUDA(cudaMemsetAsync(w.ticket, 0, 16, st));
  const int nc = m->nc, G = R.G;
  k_fcg_init<MW><<<G, kKB, 0, st>>>(R.t, R.A, b64, x64, xh, xl, rh, rl, w);
  DIFVM_TRY(check_launch("fcg_init"));
  amg_vcycle(R, 0, rh, z32, w, 1, st);
  k_fcg_p<<<G, kKB, 0, st>>>(nc, z32, ph, pl, w, 1);
  DIFVM_TRY(check_launch("fcg_p"));
  // q = A p (matrix, D, p and q as float pairs); x, r, p, q pairs; p pair and z
  const uint64_t n64 = (uint64_t)nc;
  const uint64_t fcg_bytes = lev_mat_bytes(R.H->lev[0], 4) + 20 * n64 + 48 * n64 + 20 * n64;
  count_bytes(lev_mat_bytes(R.H->lev[0], 4) + 36 * n64);   // the FP64 initial residual
  auto iter = [&](cudaStream_t s) {
    count_bytes(fcg_bytes);
    prof_before(DIFVM_PROF_PCG_SPMV, s);
    launch_pdl(k_fcg_spmv<MW>, G, kKB, s, R.t, R.A, ph, pl, qh, ql, w);
    prof_after(DIFVM_PROF_PCG_SPMV, s);
    launch_pdl(k_fcg_update, G, kKB, s, nc, ph, pl, qh, ql, xh, xl, rh, rl, w);
    amg_vcycle(R, 0, rh, z32, w, 0, s);
    launch_pdl(k_fcg_p, G, kKB, s, nc, z32, ph, pl, w, 0);
    count_launch(); count_launch(); count_launch();
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
      DIFVM_TRY(check_error("fcg_iter"));
      DIFVM_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
      DIFVM_CUDA(cudaStreamSynchronize(st));
      if (hs.done) break;
    }
  }
  k_fcg_final<<<G, kKB, 0, st>>>(nc, xh, xl, x64, w);
  DIFVM_TRY(check_launch("fcg_final"));
  if (info) {
    k_amg_info<<<1, 32, 0, st>>>(w.st, info, 0, -1);
    DIFVM_TRY(check_launch("amg_info"));
  }
  if (graph) return DIFVM_OK;
  KState hs;
  DIFVM_CUDA(cudaMemcpyAsync(&hs, w.st, sizeof(KState), cudaMemcpyDeviceToHost, st));
  DIFVM_CUDA(cudaStreamSynchronize(st));
  return (difvm_status)hs.status;
}

difvm_status amg_refine(difvm_mesh* m, const difvm_solve_opts* o, const float* D, const float* Lo,
                        const double* b64, double* x64, void* ws, size_t wsbytes, difvm_solve_info* info,
                        cudaStream_t st) {
  if (m->ell_wmax <= 4) return amg_mixed_mw<4>(m, o, D, Lo, b64, x64, ws, wsbytes, info, st);
  if (m->ell_wmax <= 8) return amg_mixed_mw<8>(m, o, D, Lo, b64, x64, ws, wsbytes, info, st);
  return amg_mixed_mw<0>(m, o, D, Lo, b64, x64, ws, wsbytes, info, st);
}

}  // namespace difvm

using namespace difvm;

extern "C" difvm_status difvm_mesh_amg_config(difvm_mesh_t m, int tail_rows, int tail_bps) {
  DIFVM_TRY(check_mesh(m));
  if (tail_rows < -1 || tail_bps < -1 || tail_bps == 0)
    return set_error(DIFVM_EINVAL, "bad multigrid configuration (%d, %d)", tail_rows, tail_bps);
  m->amg_tail_rows = tail_rows;
  m->amg_tail_bps = tail_bps;
  return DIFVM_OK;
}
