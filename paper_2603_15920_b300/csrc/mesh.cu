// Mesh ingest (host) and derived face coefficients (device).
//
// difvm_mesh_create validates the static graph arrays of Sec. 2.4.1, applies a
// reverse Cuthill-McKee cell renumbering (locality of the owner/neighbour
// gathers), orients every internal face owner < neighbour, sorts internal faces
// by (owner, neighbour), keeps boundary faces grouped by patch (sorted by owner
// inside a patch), builds the cell -> face CSR used by every deterministic
// face -> cell reduction, and computes the derived coefficients of Sec. 2.3.2
// (w_f, c_f, k_f, 1/V) in FP64 on the device, with FP32 copies for the F32 path.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>

#include <algorithm>
#include <numeric>

#include <nvtx3/nvToolsExt.h>

#include "difvm_internal.cuh"

namespace difvm {

static thread_local std::string g_err;
static std::atomic<uint64_t> g_launches{0};

difvm_status set_error(difvm_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static std::atomic<uint64_t> g_alg_bytes{0};
static thread_local bool g_bytes_paused = false;
void count_bytes(uint64_t bytes) {
  if (!g_bytes_paused) g_alg_bytes.fetch_add(bytes, std::memory_order_relaxed);
}
void count_bytes_pause(bool paused) { g_bytes_paused = paused; }

struct ProfState {
  int tag = 0;
  int cap = 0;
  int n = 0;
  uint64_t bytes = 0;
  std::vector<cudaEvent_t> ev;
};
static ProfState g_prof;

bool prof_active() { return g_prof.tag != 0; }

// phase timing of the PISO step
struct PhaseState {
  bool on = false;
  int cap = 0;
  std::vector<cudaEvent_t> ev;
  std::vector<int> ph;
  int64_t steps = 0;
};
static PhaseState g_phase;
static bool g_nvtx_open = false;
static const char* const kPhaseNames[DIFVM_PHASE_COUNT] = {
    "difvm:windkessel", "difvm:momentum_assembly", "difvm:momentum_solve", "difvm:pressure_assembly",
    "difvm:pressure_solve", "difvm:correction"};

void phase_mark(int phase, cudaStream_t s) {
  if (stream_capturing(s)) return;
  if (g_nvtx_open) nvtxRangePop();
  g_nvtx_open = phase >= 0;
  if (phase >= 0) nvtxRangePushA(kPhaseNames[phase]);
  if (!g_phase.on || (int)g_phase.ph.size() >= g_phase.cap) return;
  const size_t k = g_phase.ph.size();
  cudaEventRecord(g_phase.ev[k], s);
  g_phase.ph.push_back(phase);
  if (phase < 0) ++g_phase.steps;
}

void prof_before(int tag, cudaStream_t s) {
  if (g_prof.tag == tag && g_prof.n < g_prof.cap) cudaEventRecord(g_prof.ev[2 * g_prof.n], s);
}

void prof_bytes(int tag, uint64_t bytes) {
  if (g_prof.tag == tag && g_prof.n < g_prof.cap) g_prof.bytes += bytes;
}

void prof_after(int tag, cudaStream_t s) {
  if (g_prof.tag == tag && g_prof.n < g_prof.cap) cudaEventRecord(g_prof.ev[2 * g_prof.n++ + 1], s);
}

difvm_status check_launch(const char* what) {
  count_launch();
  return check_error(what);
}

difvm_status check_error(const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return set_error(DIFVM_ECUDA, "%s launch: %s", what, cudaGetErrorString(e));
  return DIFVM_OK;
}

difvm_status check_mesh(const difvm_mesh* m) {
  if (!m) return set_error(DIFVM_EINVAL, "null mesh handle");
  return DIFVM_OK;
}

difvm_status check_prec(difvm_prec p) {
  if (p != DIFVM_F32 && p != DIFVM_F64) return set_error(DIFVM_EINVAL, "bad precision %d", (int)p);
  return DIFVM_OK;
}

// ----------------------------------------------------------------- RCM
// Reverse Cuthill-McKee on the cell adjacency graph.  Components are handled
// in the order of their smallest cell id and each component's order is
// reversed in place, so the cells of a batched case stay contiguous and in
// case order.  Returns new_of_old.
static std::vector<int32_t> rcm(int nc, const std::vector<int>& ap, const std::vector<int>& aj) {
  std::vector<int32_t> order;
  order.reserve(nc);
  std::vector<char> vis(nc, 0);
  std::vector<int> level(nc, -1), deg(nc);
  for (int i = 0; i < nc; ++i) deg[i] = ap[i + 1] - ap[i];
  std::vector<int> q, comp, nb;
  auto bfs_levels = [&](int s, std::vector<int>& out) -> int {  // returns eccentricity
    out.clear();
    out.push_back(s);
    level[s] = 0;
    int ecc = 0;
    for (size_t h = 0; h < out.size(); ++h) {
      int u = out[h];
      for (int e = ap[u]; e < ap[u + 1]; ++e) {
        int v = aj[e];
        if (level[v] < 0) {
          level[v] = level[u] + 1;
          ecc = std::max(ecc, level[v]);
          out.push_back(v);
        }
      }
    }
    return ecc;
  };
  for (int s0 = 0; s0 < nc; ++s0) {
    if (vis[s0]) continue;
    // pseudo-peripheral start (George & Liu): repeat BFS from a min-degree
    // node of the last level while the eccentricity grows
    int s = s0;
    int ecc = bfs_levels(s, comp);
    for (int iter = 0; iter < 8; ++iter) {
      int best = -1;
      for (int u : comp)
        if (level[u] == ecc && (best < 0 || deg[u] < deg[best] || (deg[u] == deg[best] && u < best)))
          best = u;
      for (int u : comp) level[u] = -1;
      int e2 = bfs_levels(best, comp);
      if (e2 <= ecc) {
        for (int u : comp) level[u] = -1;
        bfs_levels(s, comp);
        break;
      }
      s = best;
      ecc = e2;
    }
    for (int u : comp) level[u] = -1;
    // Cuthill-McKee from s: neighbours in increasing degree (ties by id)
    size_t c0 = order.size();
    order.push_back(s);
    vis[s] = 1;
    for (size_t h = c0; h < order.size(); ++h) {
      int u = order[h];
      nb.clear();
      for (int e = ap[u]; e < ap[u + 1]; ++e)
        if (!vis[aj[e]]) nb.push_back(aj[e]);
      std::sort(nb.begin(), nb.end(), [&](int a, int b) {
        return deg[a] < deg[b] || (deg[a] == deg[b] && a < b);
      });
      for (int v : nb) {
        if (!vis[v]) {
          vis[v] = 1;
          order.push_back(v);
        }
      }
    }
    std::reverse(order.begin() + c0, order.end());
  }
  std::vector<int32_t> new_of_old(nc);
  for (int k = 0; k < nc; ++k) new_of_old[order[k]] = k;
  return new_of_old;
}

// ------------------------------------------------------------ device setup
// Derived face coefficients (Sec. 2.3.2), FP64:
//   d   = C_N - C_O (internal), x_f - C_O (boundary)
//   w_f = S.(C_N - x_f) / S.d                 owner weight of linear interpolation
//   c_f = |Delta_f| / |d|                     for the split S = Delta + k of Eq. nonortho_flux:
//         over-relaxed |S|^2 / S.d, minimum S.d / |d|^2, orthogonal and none |S| / |d|;
//         boundary faces (no cell-to-cell vector) |S|^2 / S.d for every split
//   k_f = S - c_f d                           non-orthogonal remainder (internal only; 0 for none)
__global__ void k_face_coeffs(int ni, int nf, int split, const int2* on, const int* bown, const double* Sf,
                              const double* Cf, const double* C, V4<double>* Sw64,
                              V4<double>* ck64, V4<float>* Sw32, V4<float>* ck32) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= nf) return;
  double S[3] = {Sf[3 * f], Sf[3 * f + 1], Sf[3 * f + 2]};
  double xf[3] = {Cf[3 * f], Cf[3 * f + 1], Cf[3 * f + 2]};
  int O = f < ni ? on[f].x : bown[f - ni];
  double CO[3] = {C[3 * O], C[3 * O + 1], C[3 * O + 2]};
  double SS = S[0] * S[0] + S[1] * S[1] + S[2] * S[2];
  double w = 1.0, c, k[3] = {0, 0, 0};
  if (f < ni) {
    int N = on[f].y;
    double CN[3] = {C[3 * N], C[3 * N + 1], C[3 * N + 2]};
    double d[3] = {CN[0] - CO[0], CN[1] - CO[1], CN[2] - CO[2]};
    double Sd = S[0] * d[0] + S[1] * d[1] + S[2] * d[2];
    w = (S[0] * (CN[0] - xf[0]) + S[1] * (CN[1] - xf[1]) + S[2] * (CN[2] - xf[2])) / Sd;
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (split == DIFVM_NONORTH_MINIMUM) c = Sd / dd;
    else if (split == DIFVM_NONORTH_ORTHOGONAL || split == DIFVM_NONORTH_NONE) c = sqrt(SS) / sqrt(dd);
    else c = SS / Sd;
    if (split != DIFVM_NONORTH_NONE)
      for (int a = 0; a < 3; ++a) k[a] = S[a] - c * d[a];
  } else {
    double d[3] = {xf[0] - CO[0], xf[1] - CO[1], xf[2] - CO[2]};
    c = SS / (S[0] * d[0] + S[1] * d[1] + S[2] * d[2]);
  }
  Sw64[f] = V4<double>{S[0], S[1], S[2], w};
  ck64[f] = V4<double>{c, k[0], k[1], k[2]};
  Sw32[f] = V4<float>{(float)S[0], (float)S[1], (float)S[2], (float)w};
  ck32[f] = V4<float>{(float)c, (float)k[0], (float)k[1], (float)k[2]};
}

__global__ void k_cell_coeffs(int nc, const double* V, double* rV64, float* V32, float* rV32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nc) return;
  double v = V[i];
  rV64[i] = 1.0 / v;
  V32[i] = (float)v;
  rV32[i] = (float)(1.0 / v);
}

// Sw face records in half-face slot order (zero on padding)
__global__ void k_hf_fill(int ns, const int* fid, const V4<double>* Sw64, const V4<float>* Sw32,
                          V4<double>* hsw64, V4<float>* hsw32) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ns) return;
  const int f = fid[k];
  if (f < 0) {
    hsw64[k] = V4<double>{0, 0, 0, 0};
    hsw32[k] = V4<float>{0, 0, 0, 0};
    return;
  }
  hsw64[k] = Sw64[f];
  hsw32[k] = Sw32[f];
}

// w_f of the internal faces as arrays of their own (read by face id)
__global__ void k_w_fill(int ni, const V4<double>* Sw64, double* w64, float* w32) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= ni) return;
  w64[f] = Sw64[f].w;
  w32[f] = (float)Sw64[f].w;
}

static void free_mesh(difvm_mesh* m) {
  if (!m) return;
  void* ptrs[] = {m->on,   m->bown, m->cptr, m->cent, m->bkind, m->bpatch, m->Sw64,
                  m->ck64, m->Sw32, m->ck32, m->V64,  m->rV64,  m->C64,    m->Cf64,
                  m->V32,  m->rV32, m->ell_soff, m->ell_col, m->ell_map, m->ell_c16,
                  m->seg_case, m->seg_cb0, m->seg_cs, m->hf_soff, m->hf_nb, m->hf_fid,
                  m->hf_nf, m->hf_sw64, m->hf_sw32, m->hf_cw, m->hf_fb, m->w64, m->w32};
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(m->device);
  for (void* p : ptrs)
    if (p) cudaFree(p);
  amg_free(m->amg);
  dic_free(m->dic);
  if (cur >= 0) cudaSetDevice(cur);
  delete m;
}

template <typename T>
static difvm_status upload(T** dst, const T* src, size_t n) {
  if (n == 0) n = 1;
  if (cudaMalloc((void**)dst, n * sizeof(T)) != cudaSuccess)
    return set_error(DIFVM_ENOMEM, "cudaMalloc of %zu bytes failed", n * sizeof(T));
  if (src) DIFVM_CUDA(cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
  return DIFVM_OK;
}

static difvm_status build(const difvm_mesh_desc* d, difvm_mesh* m) {
  const int nc = d->n_cells, ni = d->n_internal, nf = d->n_faces, np = d->n_patches;
  const int nb = nf - ni;
  if (nc <= 0 || ni < 0 || nf < ni || np < 0 || np > 65535)
    return set_error(DIFVM_EINVAL, "bad sizes nc=%d ni=%d nf=%d npatch=%d", nc, ni, nf, np);
  if (!d->owner || (ni > 0 && !d->neighbour) || !d->Sf || !d->Cf || !d->V || !d->C)
    return set_error(DIFVM_EINVAL, "null mesh array");
  if (d->flags & ~(uint32_t)(DIFVM_RENUMBER_RCM | DIFVM_SORT_FACES | DIFVM_NONORTH_MASK | DIFVM_WIDE_INDICES))
    return set_error(DIFVM_EINVAL, "unknown mesh flags 0x%x", d->flags);
  if (nb > 0 && (!d->patch_start || !d->patch_size || !d->patch_type))
    return set_error(DIFVM_EINVAL, "boundary faces without patches");
  if (nb > kMaxBoundaryFaces)
    return set_error(DIFVM_EINVAL, "%d boundary faces: at most %d are supported", nb, kMaxBoundaryFaces);
  for (int f = 0; f < nf; ++f)
    if (d->owner[f] < 0 || d->owner[f] >= nc)
      return set_error(DIFVM_EINVAL, "owner[%d]=%d out of range", f, d->owner[f]);
  for (int f = 0; f < ni; ++f) {
    if (d->neighbour[f] < 0 || d->neighbour[f] >= nc)
      return set_error(DIFVM_EINVAL, "neighbour[%d]=%d out of range", f, d->neighbour[f]);
    if (d->neighbour[f] == d->owner[f])
      return set_error(DIFVM_EINVAL, "face %d has owner == neighbour", f);
  }
  for (int i = 0; i < nc; ++i)
    if (!(d->V[i] > 0)) return set_error(DIFVM_EINVAL, "V[%d] = %g is not positive", i, d->V[i]);
  int expect = ni;
  for (int p = 0; p < np; ++p) {
    if (d->patch_start[p] != expect || d->patch_size[p] < 0)
      return set_error(DIFVM_EINVAL, "patch %d does not continue the boundary faces contiguously", p);
    if (d->patch_type[p] < 0 || d->patch_type[p] > 3)
      return set_error(DIFVM_EINVAL, "patch %d has bad type %d", p, d->patch_type[p]);
    expect += d->patch_size[p];
  }
  if (expect != nf) return set_error(DIFVM_EINVAL, "patches cover %d of %d faces", expect, nf);
  int ncases = d->n_cases > 1 ? d->n_cases : 1;
  m->case_start.assign(ncases + 1, 0);
  m->case_start[ncases] = nc;
  if (ncases > 1) {
    if (!d->case_cell_start) return set_error(DIFVM_EINVAL, "n_cases > 1 without case_cell_start");
    for (int k = 0; k <= ncases; ++k) m->case_start[k] = d->case_cell_start[k];
    if (m->case_start[0] != 0 || m->case_start[ncases] != nc)
      return set_error(DIFVM_EINVAL, "case_cell_start must run from 0 to n_cells");
    for (int k = 0; k < ncases; ++k)
      if (m->case_start[k + 1] <= m->case_start[k])
        return set_error(DIFVM_EINVAL, "empty or decreasing case %d", k);
    // cases must not be coupled by faces
    std::vector<int> case_of(nc);
    for (int k = 0; k < ncases; ++k)
      for (int i = m->case_start[k]; i < m->case_start[k + 1]; ++i) case_of[i] = k;
    for (int f = 0; f < ni; ++f)
      if (case_of[d->owner[f]] != case_of[d->neighbour[f]])
        return set_error(DIFVM_EINVAL, "face %d couples two cases", f);
  }
  m->nc = nc; m->ni = ni; m->nf = nf; m->nb = nb; m->npatch = np; m->ncases = ncases;
  m->patch_start.assign(d->patch_start, d->patch_start + np);
  m->patch_size.assign(d->patch_size, d->patch_size + np);
  m->patch_type.assign(d->patch_type, d->patch_type + np);

  // cell renumbering
  std::vector<int32_t> nw(nc);
  if (d->flags & DIFVM_RENUMBER_RCM) {
    std::vector<int> ap(nc + 1, 0), aj(2 * (size_t)ni);
    for (int f = 0; f < ni; ++f) { ap[d->owner[f] + 1]++; ap[d->neighbour[f] + 1]++; }
    for (int i = 0; i < nc; ++i) ap[i + 1] += ap[i];
    std::vector<int> fill(ap.begin(), ap.end() - 1);
    for (int f = 0; f < ni; ++f) {
      aj[fill[d->owner[f]]++] = d->neighbour[f];
      aj[fill[d->neighbour[f]]++] = d->owner[f];
    }
    nw = rcm(nc, ap, aj);
  } else {
    std::iota(nw.begin(), nw.end(), 0);
  }
  m->cell_new_of_old = nw;

  // internal faces: orient owner < neighbour, sort by (owner, neighbour)
  std::vector<int64_t> key(ni);
  std::vector<int8_t> flip(nf, 0);
  std::vector<int> fo(nf), fn(ni);
  for (int f = 0; f < ni; ++f) {
    int o = nw[d->owner[f]], n = nw[d->neighbour[f]];
    if (o > n) { std::swap(o, n); flip[f] = 1; }
    fo[f] = o; fn[f] = n;
    key[f] = (int64_t)o * nc + n;
  }
  std::vector<int32_t> perm(nf);
  std::iota(perm.begin(), perm.end(), 0);
  if (d->flags & DIFVM_SORT_FACES) {
    std::stable_sort(perm.begin(), perm.begin() + ni, [&](int a, int b) { return key[a] < key[b]; });
    for (int p = 0; p < np; ++p) {
      int s = d->patch_start[p], e = s + d->patch_size[p];
      std::stable_sort(perm.begin() + s, perm.begin() + e,
                       [&](int a, int b) { return nw[d->owner[a]] < nw[d->owner[b]]; });
    }
  }
  for (int f = ni; f < nf; ++f) fo[f] = nw[d->owner[f]];
  m->face_old_of_new = perm;
  m->face_flip.assign(nf, 0);
  for (int k = 0; k < nf; ++k) m->face_flip[k] = flip[perm[k]];

  // internal-order arrays
  std::vector<int2> on(ni > 0 ? ni : 1);
  std::vector<int> bown(nb > 0 ? nb : 1);
  std::vector<double> Sf(3 * (size_t)nf), Cf(3 * (size_t)nf), C(3 * (size_t)nc), V(nc);
  for (int k = 0; k < nf; ++k) {
    int f = perm[k];
    double sg = flip[f] ? -1.0 : 1.0;
    for (int a = 0; a < 3; ++a) {
      Sf[3 * (size_t)k + a] = sg * d->Sf[3 * (size_t)f + a];
      Cf[3 * (size_t)k + a] = d->Cf[3 * (size_t)f + a];
    }
    if (k < ni) on[k] = make_int2(fo[f], fn[f]);
    else bown[k - ni] = fo[f];
  }
  for (int i = 0; i < nc; ++i) {
    int j = nw[i];
    V[j] = d->V[i];
    for (int a = 0; a < 3; ++a) C[3 * (size_t)j + a] = d->C[3 * (size_t)i + a];
  }
  // geometry check: S.d > 0 on every face (owner centroid behind the face)
  for (int k = 0; k < nf; ++k) {
    int O = k < ni ? on[k].x : bown[k - ni];
    const double* S = &Sf[3 * (size_t)k];
    double dd[3];
    for (int a = 0; a < 3; ++a)
      dd[a] = (k < ni ? C[3 * (size_t)on[k].y + a] : Cf[3 * (size_t)k + a]) - C[3 * (size_t)O + a];
    if (!(S[0] * dd[0] + S[1] * dd[1] + S[2] * dd[2] > 0))
      return set_error(DIFVM_EINVAL, "face %d (input id %d): S.d <= 0", k, perm[k]);
  }
  // cell -> face CSR, ascending face id per cell (internal faces precede boundary faces)
  std::vector<int> cptr(nc + 1, 0);
  for (int k = 0; k < ni; ++k) { cptr[on[k].x + 1]++; cptr[on[k].y + 1]++; }
  for (int b = 0; b < nb; ++b) cptr[bown[b] + 1]++;
  for (int i = 0; i < nc; ++i) cptr[i + 1] += cptr[i];
  m->nnz = cptr[nc];
  std::vector<int> cent((size_t)std::max<int64_t>(m->nnz, 1));
  std::vector<int> fill(cptr.begin(), cptr.end() - 1);
  for (int k = 0; k < ni; ++k) {
    cent[fill[on[k].x]++] = (k << 1);
    cent[fill[on[k].y]++] = (k << 1) | 1;
  }
  for (int b = 0; b < nb; ++b) cent[fill[bown[b]]++] = ((ni + b) << 1);
  m->max_row = 0;
  for (int i = 0; i < nc; ++i) m->max_row = std::max(m->max_row, cptr[i + 1] - cptr[i]);
  // sliced-ELL layout of the internal-face entries (slice height 32)
  const int nsl = (nc + 31) / 32;
  std::vector<int> soff(nsl + 1, 0);
  for (int sl = 0; sl < nsl; ++sl) {
    int w = 0;
    for (int i = 32 * sl; i < std::min(nc, 32 * sl + 32); ++i) {
      int k = 0;
      for (int e = cptr[i]; e < cptr[i + 1]; ++e) k += (cent[e] >> 1) < ni;
      w = std::max(w, k);
    }
    soff[sl + 1] = soff[sl] + 32 * w;
    m->ell_wmax = std::max(m->ell_wmax, w);
  }
  // one width for all slices when padding costs little (uniform meshes): the
  // SpMV then computes slice offsets instead of loading them
  // (row-major within the uniform layout: slot = i * W + k, so a row of width 4
  // is one 16-byte load of columns and one of values)
  if ((int64_t)32 * m->ell_wmax * nsl <= (int64_t)soff[nsl] + soff[nsl] / 20) {
    for (int sl = 0; sl <= nsl; ++sl) soff[sl] = 32 * m->ell_wmax * sl;
    m->ell_w = m->ell_wmax;
  }
  const int uw = m->ell_w;
  auto slot = [&](int i, int k) { return uw > 0 ? i * uw + k : soff[i >> 5] + 32 * k + (i & 31); };
  std::vector<int> ecol((size_t)std::max(soff[nsl], 1), 0), emap((size_t)std::max(soff[nsl], 1), -1);
  for (int i = 0; i < nc; ++i) {
    const int sl = i >> 5, w = (soff[sl + 1] - soff[sl]) / 32;
    int k = 0;
    for (int e = cptr[i]; e < cptr[i + 1]; ++e) {
      const int f = cent[e] >> 1;
      if (f >= ni) continue;
      ecol[slot(i, k)] = (cent[e] & 1) ? on[f].x : on[f].y;
      emap[slot(i, k)] = cent[e];
      ++k;
    }
    for (; k < w; ++k) ecol[slot(i, k)] = i;
  }
  m->ell_nsl = nsl;
  m->ell_nslots = soff[nsl];
  // patch of every boundary face (the slot words carry its category)
  std::vector<int> bpatch_of(nb > 0 ? nb : 1, 0);
  for (int p = 0; p < np; ++p)
    for (int f = d->patch_start[p]; f < d->patch_start[p] + d->patch_size[p]; ++f) bpatch_of[f - ni] = p;
  // half-face layout: every CSR entry of a row, sliced ELL, column-major per slice
  std::vector<int> hsoff(nsl + 1, 0);
  int hwmax = 0;
  for (int sl = 0; sl < nsl; ++sl) {
    int w = 0;
    for (int i = 32 * sl; i < std::min(nc, 32 * sl + 32); ++i) w = std::max(w, cptr[i + 1] - cptr[i]);
    hsoff[sl + 1] = hsoff[sl] + 32 * w;
    hwmax = std::max(hwmax, w);
  }
  if ((int64_t)32 * hwmax * nsl <= (int64_t)hsoff[nsl] + hsoff[nsl] / 20) {
    for (int sl = 0; sl <= nsl; ++sl) hsoff[sl] = 32 * hwmax * sl;
    m->hf_w = hwmax;
  }
  m->hf_nslots = hsoff[nsl];
  std::vector<int> hnb((size_t)std::max<int64_t>(m->hf_nslots, 1), -1), hfid(hnb.size(), -1);
  for (int i = 0; i < nc; ++i) {
    for (int e = cptr[i]; e < cptr[i + 1]; ++e) {
      const int slot = hsoff[i >> 5] + 32 * (e - cptr[i]) + (i & 31);
      const int ent = cent[e], f = ent >> 1;
      hfid[slot] = f;
      hnb[slot] = f < ni ? 2 * ((ent & 1) ? on[f].x : on[f].y) + (ent & 1)
                         : -2 - (4 * (f - ni) + patch_cat(d->patch_type[bpatch_of[f - ni]]));
    }
  }
  // boundary kinds per bc class (2 bits each)
  std::vector<uint8_t> bkind(nb > 0 ? nb : 1);
  std::vector<uint16_t> bpatch(nb > 0 ? nb : 1);
  for (int p = 0; p < np; ++p) {
    const int cat = patch_cat(d->patch_type[p]);
    uint8_t code = 0;
    for (int cls = 0; cls < 4; ++cls) code |= (uint8_t)(bc_kind(cls, cat) << (2 * cls));
    for (int f = d->patch_start[p]; f < d->patch_start[p] + d->patch_size[p]; ++f) {
      bkind[f - ni] = code;
      bpatch[f - ni] = (uint16_t)p;
    }
  }

  // upload
  DIFVM_CUDA(cudaSetDevice(d->device));
  m->device = d->device;
  cudaDeviceGetAttribute(&m->num_sms, cudaDevAttrMultiProcessorCount, d->device);
  DIFVM_TRY(upload(&m->on, on.data(), on.size()));
  DIFVM_TRY(upload(&m->bown, bown.data(), bown.size()));
  DIFVM_TRY(upload(&m->cptr, cptr.data(), cptr.size()));
  DIFVM_TRY(upload(&m->cent, cent.data(), cent.size()));
  DIFVM_TRY(upload(&m->bkind, bkind.data(), bkind.size()));
  DIFVM_TRY(upload(&m->bpatch, bpatch.data(), bpatch.size()));
  DIFVM_TRY(upload(&m->ell_soff, soff.data(), soff.size()));
  DIFVM_TRY(upload(&m->ell_col, ecol.data(), ecol.size()));
  DIFVM_TRY(upload(&m->ell_map, emap.data(), emap.size()));
  const bool wide = (d->flags & DIFVM_WIDE_INDICES) != 0;
  if (uw == 4 && nc > 0 && !wide) {
    std::vector<short4> c16(nc);
    bool fits = true;
    for (int i = 0; i < nc && fits; ++i) {
      int d[4];
      for (int k = 0; k < 4; ++k) {
        d[k] = ecol[(size_t)i * 4 + k] - i;
        fits = fits && d[k] >= -32768 && d[k] <= 32767;
      }
      c16[i] = make_short4((short)d[0], (short)d[1], (short)d[2], (short)d[3]);
    }
    if (fits) DIFVM_TRY(upload(&m->ell_c16, c16.data(), c16.size()));
  }
  DIFVM_TRY(upload(&m->hf_soff, hsoff.data(), hsoff.size()));
  DIFVM_TRY(upload(&m->hf_nb, hnb.data(), hnb.size()));
  DIFVM_TRY(upload(&m->hf_fid, hfid.data(), hfid.size()));
  {
    std::vector<int2> hnf(hnb.size());
    for (size_t k = 0; k < hnb.size(); ++k) hnf[k] = make_int2(hnb[k], hfid[k]);
    DIFVM_TRY(upload(&m->hf_nf, hnf.data(), hnf.size()));
  }
  {
    // compact slot words, where every internal slot fits (see difvm::Hf)
    std::vector<int> hfb(nsl > 0 ? nsl : 1, 0), hcw(hnb.size(), -1);
    int f0 = 0;
    for (int sl = 0; sl < nsl; ++sl) {
      while (f0 < ni && on[f0].x < 32 * sl) ++f0;
      hfb[sl] = f0;
    }
    bool fits = !wide;
    for (int i = 0; i < nc && fits; ++i) {
      for (int e = cptr[i]; e < cptr[i + 1]; ++e) {
        const int slot = hsoff[i >> 5] + 32 * (e - cptr[i]) + (i & 31);
        const int f = cent[e] >> 1;
        if (f >= ni) {
          hcw[slot] = hnb[slot];
          continue;
        }
        const int dj = (hnb[slot] >> 1) - i, df = f - hfb[i >> 5];
        if (dj < -16384 || dj > 16383 || df < -32768 || df > 32767) {
          fits = false;
          break;
        }
        hcw[slot] = (int)(((unsigned)dj & 0x7fffu) << 16 | ((unsigned)df & 0xffffu));
      }
    }
    if (fits) {
      DIFVM_TRY(upload(&m->hf_cw, hcw.data(), hcw.size()));
      DIFVM_TRY(upload(&m->hf_fb, hfb.data(), hfb.size()));
    }
  }
  m->bown_host.assign(bown.begin(), bown.begin() + nb);
  if (d->case_cell_start) {
    // block tables of the segmented solvers (the case ranges survive the
    // renumbering: RCM keeps every case's cells contiguous and in case order)
    m->seg = true;
    std::vector<int> cb0(ncases + 1, 0), bcase;
    for (int k = 0; k < ncases; ++k) {
      const int nk = m->case_start[k + 1] - m->case_start[k];
      const int nbk = (nk + kSegRows - 1) / kSegRows;
      cb0[k + 1] = cb0[k] + nbk;
      for (int j = 0; j < nbk; ++j) bcase.push_back(k);
    }
    m->seg_nblk = cb0[ncases];
    DIFVM_TRY(upload(&m->seg_case, bcase.data(), bcase.size()));
    DIFVM_TRY(upload(&m->seg_cb0, cb0.data(), cb0.size()));
    DIFVM_TRY(upload(&m->seg_cs, m->case_start.data(), m->case_start.size()));
  }
  double* Sf_d = nullptr;
  DIFVM_TRY(upload(&Sf_d, Sf.data(), Sf.size()));
  DIFVM_TRY(upload(&m->Cf64, Cf.data(), Cf.size()));
  DIFVM_TRY(upload(&m->C64, C.data(), C.size()));
  DIFVM_TRY(upload(&m->V64, V.data(), V.size()));
  DIFVM_TRY(upload<V4<double>>(&m->Sw64, nullptr, nf));
  DIFVM_TRY(upload<V4<double>>(&m->ck64, nullptr, nf));
  DIFVM_TRY(upload<V4<float>>(&m->Sw32, nullptr, nf));
  DIFVM_TRY(upload<V4<float>>(&m->ck32, nullptr, nf));
  DIFVM_TRY(upload<double>(&m->rV64, nullptr, nc));
  DIFVM_TRY(upload<float>(&m->V32, nullptr, nc));
  DIFVM_TRY(upload<float>(&m->rV32, nullptr, nc));
  k_face_coeffs<<<blocks_for(nf, 256), 256>>>(ni, nf, (int)(d->flags & DIFVM_NONORTH_MASK), m->on, m->bown,
                                               Sf_d, m->Cf64, m->C64,
                                               m->Sw64, m->ck64, m->Sw32, m->ck32);
  DIFVM_TRY(check_launch("face_coeffs"));
  k_cell_coeffs<<<blocks_for(nc, 256), 256>>>(nc, m->V64, m->rV64, m->V32, m->rV32);
  DIFVM_TRY(check_launch("cell_coeffs"));
  {
    const size_t ns = (size_t)std::max<int64_t>(m->hf_nslots, 1);
    DIFVM_TRY(upload<V4<double>>(&m->hf_sw64, nullptr, ns));
    DIFVM_TRY(upload<V4<float>>(&m->hf_sw32, nullptr, ns));
    k_hf_fill<<<blocks_for((int64_t)ns, 256), 256>>>((int)ns, m->hf_fid, m->Sw64, m->Sw32, m->hf_sw64,
                                                     m->hf_sw32);
    DIFVM_TRY(check_launch("hf_fill"));
    DIFVM_TRY(upload<double>(&m->w64, nullptr, std::max(ni, 1)));
    DIFVM_TRY(upload<float>(&m->w32, nullptr, std::max(ni, 1)));
    if (ni > 0) {
      k_w_fill<<<blocks_for(ni, 256), 256>>>(ni, m->Sw64, m->w64, m->w32);
      DIFVM_TRY(check_launch("w_fill"));
    }
  }
  DIFVM_CUDA(cudaDeviceSynchronize());
  cudaFree(Sf_d);
  return DIFVM_OK;
}

}  // namespace difvm

using namespace difvm;

extern "C" difvm_status difvm_mesh_create(const difvm_mesh_desc* desc, difvm_mesh_t* out) {
  if (!desc || !out) return set_error(DIFVM_EINVAL, "null argument");
  *out = nullptr;
  difvm_mesh* m = new (std::nothrow) difvm_mesh();
  if (!m) return set_error(DIFVM_ENOMEM, "host allocation failed");
  m->device = desc->device;
  difvm_status st = build(desc, m);
  if (st != DIFVM_OK) {
    free_mesh(m);
    return st;
  }
  *out = m;
  return DIFVM_OK;
}

extern "C" difvm_status difvm_mesh_permutation(difvm_mesh_t m, int32_t* cell_new_of_old,
                                               int32_t* face_old_of_new, int8_t* face_flip) {
  DIFVM_TRY(check_mesh(m));
  if (cell_new_of_old) std::copy(m->cell_new_of_old.begin(), m->cell_new_of_old.end(), cell_new_of_old);
  if (face_old_of_new) std::copy(m->face_old_of_new.begin(), m->face_old_of_new.end(), face_old_of_new);
  if (face_flip) std::copy(m->face_flip.begin(), m->face_flip.end(), face_flip);
  return DIFVM_OK;
}

extern "C" difvm_status difvm_mesh_info(difvm_mesh_t m, int64_t out[6]) {
  DIFVM_TRY(check_mesh(m));
  if (!out) return set_error(DIFVM_EINVAL, "null output");
  out[0] = m->nc; out[1] = m->ni; out[2] = m->nf; out[3] = m->nb; out[4] = m->npatch;
  out[5] = m->nnz;
  return DIFVM_OK;
}

extern "C" difvm_status difvm_mesh_layout(difvm_mesh_t m, int32_t out[2]) {
  DIFVM_TRY(check_mesh(m));
  if (!out) return set_error(DIFVM_EINVAL, "null output");
  out[0] = m->hf_cw != nullptr;
  out[1] = m->ell_c16 != nullptr;
  return DIFVM_OK;
}

extern "C" void difvm_mesh_destroy(difvm_mesh_t m) { free_mesh(m); }

extern "C" const char* difvm_last_error(void) { return g_err.c_str(); }

extern "C" uint64_t difvm_launch_count(void) { return g_launches.load(); }

extern "C" uint64_t difvm_alg_bytes(void) { return g_alg_bytes.load(); }

extern "C" uint64_t difvm_prof_bytes(void) { return g_prof.bytes; }

extern "C" difvm_status difvm_phase_prof_start(int max_marks) {
  if (max_marks <= 0) return set_error(DIFVM_EINVAL, "bad phase-profiling request");
  if (g_phase.on) return set_error(DIFVM_EINVAL, "phase profiling already active");
  g_phase.ev.resize((size_t)max_marks);
  for (auto& e : g_phase.ev) DIFVM_CUDA(cudaEventCreate(&e));
  g_phase.ph.clear();
  g_phase.cap = max_marks;
  g_phase.steps = 0;
  g_phase.on = true;
  return DIFVM_OK;
}

extern "C" difvm_status difvm_phase_prof_stop(double* ms, int64_t* steps) {
  if (!g_phase.on) return set_error(DIFVM_EINVAL, "phase profiling not active");
  difvm_status st = DIFVM_OK;
  double tot[DIFVM_PHASE_COUNT] = {0};
  for (size_t k = 0; k + 1 < g_phase.ph.size(); ++k) {
    if (g_phase.ph[k] < 0) continue;   // between steps
    float t = 0.f;
    if (cudaEventSynchronize(g_phase.ev[k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&t, g_phase.ev[k], g_phase.ev[k + 1]) != cudaSuccess) {
      st = set_error(DIFVM_ECUDA, "phase timing failed");
      break;
    }
    tot[g_phase.ph[k]] += t;
  }
  if (ms)
    for (int p = 0; p < DIFVM_PHASE_COUNT; ++p) ms[p] = tot[p];
  if (steps) *steps = g_phase.steps;
  for (auto& e : g_phase.ev) cudaEventDestroy(e);
  g_phase.ev.clear();
  g_phase.ph.clear();
  g_phase.on = false;
  return st;
}

extern "C" difvm_status difvm_prof_start(int tag, int max_launches) {
  if (tag <= 0 || max_launches <= 0) return set_error(DIFVM_EINVAL, "bad profiling request");
  if (g_prof.tag != 0) return set_error(DIFVM_EINVAL, "profiling already active");
  g_prof.ev.resize(2 * (size_t)max_launches);
  for (auto& e : g_prof.ev) DIFVM_CUDA(cudaEventCreate(&e));
  g_prof.cap = max_launches;
  g_prof.n = 0;
  g_prof.bytes = 0;
  g_prof.tag = tag;
  return DIFVM_OK;
}

extern "C" difvm_status difvm_prof_stop(double* total_ms, int64_t* launches) {
  if (g_prof.tag == 0) return set_error(DIFVM_EINVAL, "profiling not active");
  double tot = 0.0;
  difvm_status st = DIFVM_OK;
  for (int k = 0; k < g_prof.n; ++k) {
    float ms = 0.f;
    if (cudaEventSynchronize(g_prof.ev[2 * k + 1]) != cudaSuccess ||
        cudaEventElapsedTime(&ms, g_prof.ev[2 * k], g_prof.ev[2 * k + 1]) != cudaSuccess) {
      st = set_error(DIFVM_ECUDA, "event timing failed");
      break;
    }
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = g_prof.n;
  for (auto& e : g_prof.ev) cudaEventDestroy(e);
  g_prof.ev.clear();
  g_prof.tag = 0;
  g_prof.cap = g_prof.n = 0;
  return st;
}
