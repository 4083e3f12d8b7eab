// C ABI of the CGKS library: device buffers, V-cycle orchestration on the
// caller's stream, CUDA-graph capture and replay.  See include/cgks.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cmath>
#include <cstring>
#include <map>
#include <memory>
#include <stdexcept>
#include <string>
#include <vector>

#include "cgks.h"
#include "host_mesh.hpp"
#include "kernels.cuh"
#include "mlp.cuh"
#include "mlp_tc.cuh"

namespace cgks {
namespace {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct ArgError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct StateError : std::runtime_error {
  using std::runtime_error::runtime_error;
};
struct TimeoutError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define CK(x)                                                                                     \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) throw CudaError(std::string(#x) + ": " + cudaGetErrorString(e_));     \
  } while (0)

inline unsigned blocks_for(int64_t n, int b = kBlock) { return (unsigned)((n + b - 1) / b); }

// owning device allocation
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() {
    if (p) cudaFree(p);
  }
  void alloc(size_t b) {
    if (p) { cudaFree(p); p = nullptr; }
    bytes = b;
    if (b) CK(cudaMalloc(&p, b));
  }
  template <class T>
  T* as() const { return (T*)p; }
};

template <class T>
T* upload(std::vector<std::unique_ptr<DBuf>>& pool, const std::vector<T>& v) {
  pool.emplace_back(new DBuf);
  DBuf& b = *pool.back();
  b.alloc(std::max<size_t>(1, v.size()) * sizeof(T));
  if (!v.empty()) CK(cudaMemcpy(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return b.as<T>();
}
template <class T>
T* dalloc(std::vector<std::unique_ptr<DBuf>>& pool, size_t n) {
  pool.emplace_back(new DBuf);
  pool.back()->alloc(std::max<size_t>(1, n) * sizeof(T));
  CK(cudaMemset(pool.back()->p, 0, std::max<size_t>(1, n) * sizeof(T)));
  return pool.back()->as<T>();
}
template <class A>
std::vector<int32_t> to_i32(const std::vector<A>& v) {
  std::vector<int32_t> o(v.size());
  for (size_t i = 0; i < v.size(); ++i) o[i] = (int32_t)v[i];
  return o;
}

struct LevelDev {
  int n = 0, n_colors = 0;
  std::vector<int> color_off;  // host
  Topo topo{};
  int* iperm = nullptr;  // new -> original
  double* vol = nullptr;
  double *W = nullptr, *W0 = nullptr, *alpha = nullptr, *R = nullptr, *P = nullptr, *Rstar = nullptr;
  double* Wb = nullptr;  // the state's second buffer: coarse smoothing steps alternate W -> Wb -> W
  double* ones = nullptr;   // DF = 1 everywhere (prolongation ablation)
  double* relax = nullptr;  // the constant that stands for DF in LU-SGS when df_relax != 1
  FaceSet faces{};
  double* Fc = nullptr;     // coarse face fluxes [nf][nv]
  double* rface = nullptr;  // spectral radius per face [nf]
  double *D = nullptr, *dte = nullptr, *dti = nullptr;
  double *dWs64 = nullptr, *dW64 = nullptr;
  float *dWs32 = nullptr, *dW32 = nullptr;
  int* parent = nullptr;  // this level's cell -> next coarser level cell
  int *ch_off = nullptr, *ch_idx = nullptr;  // children in the finer level
};

enum BlockClass { B_RECON = 0, B_FLUX, B_GATHER, B_SWEEP, B_FACE, B_CELL, B_UPDATE };

struct MeshDev {
  int dim = 0, nv = 0, nlev = 0;
  Hierarchy H;
  bool has_hierarchy = false, has_state = false;
  std::vector<std::unique_ptr<DBuf>> pool;
  DevFine fine{};
  double *G = nullptr, *coef = nullptr, *Fface = nullptr, *Wface = nullptr, *aface = nullptr;
  dword* coef_dw = nullptr;  // double-word copy of coef for the FP32-pipe flux (flux_precision 1)
  double *gradnew = nullptr, *norm_part = nullptr, *last_norm = nullptr, *hist = nullptr;
  double* stage = nullptr;  // staging for permuted I/O, size n * max(nv*dim, ncoef*nv)
  size_t stage_elems = 0;
  int* cycle = nullptr;
  int max_hist = 0;
  int norm_blocks = 0;
  double* winf = nullptr;
  std::vector<double> winf_h;
  Counters* cnt = nullptr;
  std::vector<LevelDev> lev;
  cudaGraphExec_t graph[3][2] = {{nullptr, nullptr}, {nullptr, nullptr}, {nullptr, nullptr}};  // [plain, learned, judge][prec]
  int graph_kernels[3][2] = {{0, 0}, {0, 0}, {0, 0}};
  // learned correction buffers (fine level, colour order)
  std::vector<std::unique_ptr<DBuf>> lpool;
  __nv_bfloat16* X = nullptr;
  float *Pl = nullptr, *Yl = nullptr;
  float* Sl = nullptr;  // per-cell defect scale of the inputs and target (learned_scale 1)
  double *Wsave = nullptr, *judge_part = nullptr, *judge_out = nullptr;
  double *Rp1 = nullptr, *Rp2 = nullptr;  // restricted fine residual on levels 1 and 2 (network inputs)
  // learned-cycle policy statistics
  // learned, plain, judge, fallbacks, disabled, last judge error, then that error per variable
  double lstats[10] = {0, 0, 0, 0, 0, -1, -1, -1, -1, -1};
  // batched members (groups of cells with their own free stream)
  int n_groups = 1;
  std::vector<std::unique_ptr<DBuf>> gpool;
  std::vector<int*> lgrp;  // per level: group of each cell (device), empty if ungrouped
  double* qcell = nullptr;
  int *goff = nullptr, *gidx = nullptr, *active = nullptr;
  double *hist_g = nullptr, *last_g = nullptr;
  std::vector<int> gcount;
  // launch block sizes per kernel class (autotuned)
  int blk[7] = {256, 256, 256, 256, 128, 128, 256};
  void drop_graphs() {
    for (auto& k : graph)
      for (auto& g : k)
        if (g) { cudaGraphExecDestroy(g); g = nullptr; }
  }
  ~MeshDev() { drop_graphs(); }
};

}  // namespace
}  // namespace cgks

namespace cgks {
namespace {
// learned-correction network state (one per context)
struct MlpState {
  bool ready = false;
  std::vector<std::unique_ptr<DBuf>> pool;   // parameters and optimiser state
  std::vector<std::unique_ptr<DBuf>> work;   // batch-sized work buffers
  int64_t work_rows = 0;
  float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;
  __nv_bfloat16* theta_bf = nullptr;
  int step = 0;
  // forward implementation: 0 = fused tcgen05 kernel (tensor memory), 1 = mma.sync GEMM chain
  int impl = 0;
  int* tc_err = nullptr;  // set by the tcgen05 kernel if a bounded wait gave up
  bool tc_attr = false;   // dynamic shared-memory size set for the tcgen05 kernel
  int tc_blocks = 0;      // resident CTAs of the (persistent) tcgen05 kernel on the device
  // work buffers (rows = work_rows)
  float *Z1 = nullptr, *Z2 = nullptr, *P = nullptr, *dP = nullptr, *part = nullptr, *loss = nullptr;
  __nv_bfloat16 *A1 = nullptr, *A2 = nullptr, *dPb = nullptr, *dZ2 = nullptr, *dZ1 = nullptr;
  __nv_bfloat16* Xb = nullptr;
  float* Yb = nullptr;
  int* idx = nullptr;
  float* split = nullptr;  // split-K partials
  size_t split_elems = 0;
  // training set (rows of 76 bf16 features and 4 fp32 targets)
  std::vector<std::unique_ptr<DBuf>> data;
  __nv_bfloat16* X = nullptr;
  float* Y = nullptr;
  int64_t rows = 0, cap = 0;
};
}  // namespace
}  // namespace cgks

struct cgks_ctx {
  cgks_config cfg{};
  cgks::MlpState mlp;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::map<int, std::unique_ptr<cgks::MeshDev>> meshes;
  std::string err;
  std::vector<std::unique_ptr<cgks::DBuf>> scratch;  // point-evaluation helpers
  int sms = 148;                                      // SM count of the device (set at creation)
  int device = 0;                                     // device current at creation; all work runs there
  double* noalloc_scratch = nullptr;                  // device address of the no-allocation scratch array
  int cluster_cs[2] = {0, 0};  // blocks per cluster of the 2-D coarse-step cluster kernel [FP64, FP32]; 0: none
  // pinned host buffer for the small per-chunk reads of cgks_vcycle
  double* pin = nullptr;
  size_t pin_cap = 0;
  cgks::DBuf pack;  // its device counterpart
};

namespace cgks {
namespace {

MeshDev& get_mesh(cgks_t* h, int id) {
  auto it = h->meshes.find(id);
  if (it == h->meshes.end()) throw ArgError("unknown mesh id " + std::to_string(id));
  return *it->second;
}

PhysParams phys(const cgks_config& c, int dim) { return make_phys(c.gamma, dim, c.tau_c1, c.tau_c2, c.mu); }

// Block size for a launch over n items: the (tuned) size b, halved down to one
// warp while the grid would give fewer than two blocks per SM, so that the
// small coarse-level and per-colour launches spread over every SM.
int fit_block(const cgks_t* h, int64_t n, int b) {
  while (b > 32 && (n + b - 1) / b < 2 * (int64_t)h->sms) b >>= 1;
  return b;
}

// ---- device structures from the host hierarchy ----------------------------
void build_fine_device(MeshDev& M) {
  const FineLevel& F = M.H.fine;
  const int dim = F.dim, nfc = F.nfc;
  const int64_t n = F.n;
  auto& P = M.pool;
  DevFine d{};
  d.n = (int)n;
  d.nf = (int)F.nf;
  d.fL = upload(P, to_i32(F.fL));
  d.fR = upload(P, to_i32(F.fR));
  d.ftag = upload(P, F.ftag);
  d.fn = upload(P, F.fn);
  d.fS = upload(P, F.fS);
  d.XL = upload(P, F.XL);
  d.XR = upload(P, F.XR);
  d.cface = upload(P, to_i32(F.cface));
  std::vector<signed char> cs(F.cside.begin(), F.cside.end());
  d.cside = upload(P, cs);
  d.cnbr = upload(P, to_i32(F.cnbr));
  // variable-major per-cell geometry
  auto transpose = [&](const std::vector<double>& a, int w) {
    std::vector<double> t((size_t)w * n);
    for (int64_t c = 0; c < n; ++c)
      for (int k = 0; k < w; ++k) t[(size_t)k * n + c] = a[(size_t)c * w + k];
    return t;
  };
  d.op = upload(P, transpose(F.op, F.nop));
  std::vector<unsigned char> ok(F.op_ok.begin(), F.op_ok.end());
  d.op_ok = upload(P, ok);
  d.avg0 = upload(P, transpose(F.avg0, F.nk));
  d.gg = upload(P, transpose(F.gg, nfc * dim));
  d.m2 = upload(P, transpose(F.m2, dim * dim));
  d.vol = upload(P, F.vol);
  std::vector<double> bsc(n);
  for (int64_t c = 0; c < n; ++c) bsc[c] = std::pow(F.vol[c], 2.0 / dim);
  d.bsc = upload(P, bsc);
  // per cell, the largest |monomial| of X = x - centroid over its face Gauss
  // points, in the coefficient order of the reconstruction (X_d, then X_a X_b)
  {
    const int ngp = F.ngp, nk = F.nk, nq = nk - dim;
    const int qa[6] = {0, 0, 0, 1, 1, 2}, qb[6] = {0, 1, 2, 1, 2, 2};
    const int qa2[3] = {0, 0, 1}, qb2[3] = {0, 1, 1};
    std::vector<double> gm((size_t)nk * n, 0.0);
    for (int64_t c = 0; c < n; ++c)
      for (int k = 0; k < (F.mixed ? (int)F.cnf[c] : nfc); ++k) {
        const int64_t f = F.cface[c * nfc + k];
        const std::vector<double>& X = F.cside[c * nfc + k] > 0 ? F.XL : F.XR;
        for (int g = 0; g < (F.mixed ? (int)F.fngp[f] : ngp); ++g) {
          const double* x = &X[((size_t)f * ngp + g) * dim];
          for (int d = 0; d < dim; ++d) {
            double& t = gm[(size_t)d * n + c];
            t = std::max(t, std::fabs(x[d]));
          }
          for (int q = 0; q < nq; ++q) {
            const int a = dim == 2 ? qa2[q] : qa[q], b = dim == 2 ? qb2[q] : qb[q];
            double& t = gm[(size_t)(dim + q) * n + c];
            t = std::max(t, std::fabs(x[a] * x[b]));
          }
        }
      }
    d.gpmax = upload(P, gm);
  }
  if (F.mixed) {
    std::vector<signed char> cnf(F.cnf.begin(), F.cnf.end()), fngp(F.fngp.begin(), F.fngp.end());
    d.cnf = upload(P, cnf);
    d.fngp = upload(P, fngp);
    d.gw = upload(P, F.gw);
  }
  M.fine = d;
}

Topo make_topo(MeshDev& M, int64_t n, const std::vector<int64_t>& off, const std::vector<int64_t>& nbr,
               const std::vector<int32_t>& tag, const std::vector<int8_t>& side, const std::vector<double>& S,
               const std::vector<double>& nrm, const double* vol_dev, const std::vector<int64_t>& face) {
  auto& P = M.pool;
  Topo t{};
  t.n = (int)n;
  t.off = upload(P, to_i32(off));
  t.nbr = upload(P, to_i32(nbr));
  t.tag = upload(P, tag);
  std::vector<signed char> sd(side.begin(), side.end());
  t.side = upload(P, sd);
  t.S = upload(P, S);
  t.nrm = upload(P, nrm);
  t.vol = vol_dev;
  t.face = upload(P, to_i32(face));
  return t;
}

// The factor that replaces DF in the LU-SGS relaxation when df_relax != 1:
// 1 for the fully implicit scheme, relax_beta for the fixed-factor scheme.
double relax_constant(const cgks_config& cfg) { return cfg.df_relax == 2 ? cfg.relax_beta : 1.0; }

void alloc_level_state(MeshDev& M, LevelDev& L, const cgks_config& cfg) {
  auto& P = M.pool;
  const int nv = M.nv;
  L.W = dalloc<double>(P, (size_t)L.n * nv);
  L.Wb = dalloc<double>(P, (size_t)L.n * nv);
  L.W0 = dalloc<double>(P, (size_t)L.n * nv);
  L.alpha = dalloc<double>(P, L.n);
  L.ones = upload(P, std::vector<double>(L.n, 1.0));
  L.relax = upload(P, std::vector<double>(L.n, relax_constant(cfg)));
  L.R = dalloc<double>(P, (size_t)L.n * nv);
  L.P = dalloc<double>(P, (size_t)L.n * nv);
  L.Rstar = dalloc<double>(P, (size_t)L.n * nv);
  L.D = dalloc<double>(P, L.n);
  L.dte = dalloc<double>(P, L.n);
  L.dti = dalloc<double>(P, L.n);
  L.dWs64 = dalloc<double>(P, (size_t)L.n * nv);
  L.dW64 = dalloc<double>(P, (size_t)L.n * nv);
  L.dWs32 = dalloc<float>(P, (size_t)L.n * nv);
  L.dW32 = dalloc<float>(P, (size_t)L.n * nv);
}

void build_levels_device(MeshDev& M, const cgks_config& cfg) {
  const FineLevel& F = M.H.fine;
  const int dim = F.dim, nfc = F.nfc;
  M.lev.clear();
  M.lev.resize(1 + M.H.coarse.size());
  // fine level
  {
    LevelDev& L = M.lev[0];
    L.n = (int)F.n;
    L.n_colors = F.n_colors;
    L.color_off.assign(F.color_off.begin(), F.color_off.end());
    L.iperm = upload(M.pool, to_i32(F.iperm));
    L.vol = const_cast<double*>(M.fine.vol);
    std::vector<int64_t> off(F.n + 1), nbr(F.n * nfc), face(F.n * nfc);
    std::vector<int32_t> tag(F.n * nfc);
    std::vector<int8_t> side(F.n * nfc);
    std::vector<double> S(F.n * nfc), nrm(F.n * nfc * dim);
    // cell -> face entries (CSR); a mixed mesh's cells have 4 to 6 faces
    off[0] = 0;
    for (int64_t c = 0; c < F.n; ++c) off[c + 1] = off[c] + (F.mixed ? (int)F.cnf[c] : nfc);
    const int64_t ne = off[F.n];
    nbr.resize(ne); face.resize(ne); tag.resize(ne); side.resize(ne); S.resize(ne); nrm.resize(ne * dim);
    for (int64_t c = 0; c < F.n; ++c)
      for (int64_t e = off[c]; e < off[c + 1]; ++e) {
        const int64_t k = c * nfc + (e - off[c]), f = F.cface[k];
        nbr[e] = F.cnbr[k];
        face[e] = f;
        tag[e] = F.ftag[f];
        side[e] = F.cside[k];
        S[e] = F.fS[f];
        for (int d = 0; d < dim; ++d) nrm[e * dim + d] = F.cside[k] * F.fn[f * dim + d];
      }
    L.topo = make_topo(M, F.n, off, nbr, tag, side, S, nrm, L.vol, face);
    alloc_level_state(M, L, cfg);
    L.faces = FaceSet{M.fine.nf, M.fine.fL, M.fine.fR, M.fine.ftag, M.fine.fn, M.fine.fS};
    L.rface = dalloc<double>(M.pool, F.nf);
  }
  for (size_t l = 0; l < M.H.coarse.size(); ++l) {
    const CoarseLevel& C = M.H.coarse[l];
    LevelDev& L = M.lev[l + 1];
    L.n = (int)C.n;
    L.n_colors = C.n_colors;
    L.color_off.assign(C.color_off.begin(), C.color_off.end());
    L.iperm = upload(M.pool, to_i32(C.iperm));
    L.vol = upload(M.pool, C.vol);
    const int64_t ne = C.cf_off[C.n];
    std::vector<int64_t> nbr(ne);
    std::vector<int32_t> tag(ne);
    std::vector<double> S(ne), nrm(ne * dim);
    for (int64_t J = 0; J < C.n; ++J)
      for (int64_t e = C.cf_off[J]; e < C.cf_off[J + 1]; ++e) {
        const int64_t f = C.cf_face[e];
        (void)f;
        const int sd = C.cf_side[e];
        nbr[e] = sd > 0 ? C.fR[f] : C.fL[f];
        tag[e] = C.ftag[f];
        S[e] = C.fS[f];
        for (int d = 0; d < dim; ++d) nrm[e * dim + d] = sd * C.fn[f * dim + d];
      }
    L.topo = make_topo(M, C.n, C.cf_off, nbr, tag, C.cf_side, S, nrm, L.vol, C.cf_face);
    alloc_level_state(M, L, cfg);
    L.faces = FaceSet{(int)C.nf, upload(M.pool, to_i32(C.fL)), upload(M.pool, to_i32(C.fR)), upload(M.pool, C.ftag),
                      upload(M.pool, C.fn), upload(M.pool, C.fS)};
    L.Fc = dalloc<double>(M.pool, (size_t)C.nf * M.nv);
    L.rface = dalloc<double>(M.pool, C.nf);
    L.ch_off = upload(M.pool, to_i32(C.ch_off));
    L.ch_idx = upload(M.pool, to_i32(C.ch_idx));
    M.lev[l].parent = upload(M.pool, to_i32(C.parent_of_fine));
  }
  // fine-only buffers
  const int nv = M.nv, nc = dim == 2 ? 6 : 10;
  auto& P = M.pool;
  M.G = dalloc<double>(P, (size_t)F.n * nv * dim);
  M.coef = dalloc<double>(P, (size_t)F.n * nv * nc);
  if (cfg.flux_precision == 1) M.coef_dw = dalloc<dword>(P, (size_t)F.n * nv * nc);
  M.Fface = dalloc<double>(P, (size_t)F.nf * nv);
  M.Wface = dalloc<double>(P, (size_t)F.nf * nv);
  M.aface = dalloc<double>(P, F.nf);
  M.gradnew = dalloc<double>(P, (size_t)F.n * nv * dim);
  M.norm_blocks = (int)blocks_for(F.n);
  M.norm_part = dalloc<double>(P, (size_t)M.norm_blocks * 2 * nv);
  M.last_norm = dalloc<double>(P, 2 * nv);
  M.max_hist = 1 << 16;
  M.hist = dalloc<double>(P, (size_t)M.max_hist * 2 * nv);
  M.cycle = dalloc<int>(P, 1);
  M.stage_elems = (size_t)F.n * std::max(nv * dim, nv * nc);
  M.stage = dalloc<double>(P, M.stage_elems);
  M.cnt = dalloc<Counters>(P, 1);
  M.winf = dalloc<double>(P, nv);
  if (!M.winf_h.empty()) CK(cudaMemcpy(M.winf, M.winf_h.data(), nv * sizeof(double), cudaMemcpyHostToDevice));
}

// ---- kernels sequences ------------------------------------------------------
// Grid of a kernel whose warps loop over tasks: the blocks of size bs that are
// resident at once, at most nb (the grid of one task per warp).
template <typename K>
int resident_blocks(cgks_t* h, K kern, int bs, int64_t nb) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, bs, 0) != cudaSuccess || occ < 1) {
    (void)cudaGetLastError();
    return (int)nb;
  }
  return (int)std::min<int64_t>(nb, (int64_t)occ * h->sms);
}

template <int DIM>
void launch_recon(cgks_t* h, MeshDev& M) {
  LevelDev& L = M.lev[0];
  const int bs = M.blk[B_RECON];
  const int64_t nb = blocks_for(L.n, bs);  // 3-D: one thread per cell; 2-D: the kernel loops
  if constexpr (DIM == 3) {
    if (M.H.fine.mixed) {  // hexahedra, prisms, pyramids: per-cell face counts
      k_recon<3, 1><<<(int)nb, bs, 0, h->stream>>>(M.fine, L.W, M.G, L.alpha, M.winf, h->cfg.gamma, h->cfg.cfl_exp,
                                                   h->cfg.cfl_imp, h->cfg.weno_gamma_high, h->cfg.weno_eps, M.coef,
                                                   L.dte, L.dti, M.cnt, M.coef_dw);
      return;
    }
  }
  k_recon<DIM><<<DIM == 2 ? resident_blocks(h, k_recon<DIM>, bs, nb) : (int)nb, bs, 0, h->stream>>>(
      M.fine, L.W, M.G, L.alpha, M.winf, h->cfg.gamma, h->cfg.cfl_exp, h->cfg.cfl_imp, h->cfg.weno_gamma_high,
      h->cfg.weno_eps, M.coef, L.dte, L.dti, M.cnt, M.coef_dw);
}

template <int DIM>
void launch_flux(cgks_t* h, MeshDev& M, bool point = true, bool radius = true) {
  LevelDev& L = M.lev[0];
  constexpr int NGP = Dims<DIM>::NGP, FPW = 32 / NGP;
  const int64_t warps = (M.fine.nf + FPW - 1) / FPW;
  const int64_t threads = warps * 32;
  const int bs = M.blk[B_FLUX];
  const int nb = blocks_for(threads, bs);
  const PhysParams P = phys(h->cfg, DIM);
  // the FP64 kernel loops over its tasks: launch only the blocks that fit at
  // once; the double-word kernel takes one task per warp (the full grid)
  if (h->cfg.flux_precision == 1) {
    auto kern = point ? k_flux<DIM, true, dword> : k_flux<DIM, false, dword>;
    // One task per warp.  When the grid's last wave of resident blocks is
    // less than 95 % full (few waves: the 2-D meshes), take the block size of
    // 2..8 warps that fills it best among those that keep at least 3/4 of the
    // resident warps; with many waves the tail does not matter.
    auto fill_of = [&](int w, int& occ, int64_t& blocks) {
      occ = 0;
      if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, 32 * w, 0) != cudaSuccess || occ < 1) {
        (void)cudaGetLastError();
        return -1.0;
      }
      blocks = (warps + w - 1) / w;
      const double waves = (double)blocks / ((double)occ * h->sms);
      return waves / std::ceil(waves);
    };
    int bw = bs;
    int64_t bn = nb;
    int occ_def = 0;
    int64_t blk_def = 0;
    const int w_def = bs / 32;
    double best = fill_of(w_def, occ_def, blk_def);
    if (best >= 0.0 && best < 0.95) {
      for (int w = 8; w >= 2; --w) {
        int occ = 0;
        int64_t blocks = 0;
        const double fill = fill_of(w, occ, blocks);
        if (fill > best + 1e-9 && 4 * occ * w >= 3 * occ_def * w_def) {
          best = fill;
          bw = 32 * w;
          bn = blocks;
        }
      }
    }
    kern<<<(unsigned)bn, bw, 0, h->stream>>>(M.fine, M.coef_dw, L.dte, M.winf, phys_dword(P), P.gamma, M.Fface,
                                              M.Wface, M.aface, L.W, radius ? L.rface : nullptr);
  } else {
    auto kern = point ? k_flux<DIM, true, double> : k_flux<DIM, false, double>;
    if constexpr (DIM == 3) {
      if (M.H.fine.mixed) kern = point ? k_flux<3, true, double, 1> : k_flux<3, false, double, 1>;
    }
    kern<<<resident_blocks(h, kern, bs, nb), bs, 0, h->stream>>>(
        M.fine, M.coef, L.dte, M.winf, P, P.gamma, M.Fface, M.Wface, M.aface, L.W, radius ? L.rface : nullptr);
  }
}

// fine residual: slopes_update -> G <- alpha * grad_new; want_diag -> LU-SGS D;
// want_norm -> norm partials + final (hist when record)
// TS: precision of a fused forward LU-SGS step of colour 0 (fuse_c0), as in sweeps<DIM, TS>
template <int DIM, typename TS = double>
void fine_residual(cgks_t* h, MeshDev& M, bool slopes_update, bool want_diag, bool want_norm, bool record,
                   double* alpha_out_dev, double* gradnew_dev, bool fuse_c0 = false) {
  LevelDev& L = M.lev[0];
  launch_recon<DIM>(h, M);
  // the time-evolved point values only feed the slopes, the spectral radii only the LU-SGS diagonal
  launch_flux<DIM>(h, M, slopes_update || gradnew_dev != nullptr, want_diag);
  const bool grouped = !M.lgrp.empty();
  // norm partials need whole blocks of kBlock threads
  const int gb = (want_norm && !grouped) ? kBlock : M.blk[B_GATHER];
  const bool fuse = fuse_c0 && want_diag;
  TS* dWs0 = fuse ? (sizeof(TS) == 8 ? (TS*)L.dWs64 : (TS*)L.dWs32) : nullptr;
  TS* dW0 = fuse && L.n_colors == 1 ? (sizeof(TS) == 8 ? (TS*)L.dW64 : (TS*)L.dW32) : nullptr;
  auto gather = k_gather<DIM, TS>;
  if constexpr (DIM == 3) {
    if (M.H.fine.mixed) gather = k_gather<3, TS, 1>;  // per-cell face counts
  }
  gather<<<blocks_for(L.n, gb), gb, 0, h->stream>>>(
      M.fine, L.topo, M.Fface, M.Wface, M.aface, L.W, M.winf, h->cfg.gamma, L.dte, L.dti, L.R,
      slopes_update ? M.G : nullptr, alpha_out_dev ? alpha_out_dev : L.alpha, want_diag ? L.D : nullptr,
      gradnew_dev, (want_norm && !grouped) ? M.norm_part : nullptr, h->cfg.df_relax == 1 ? -1.0 : relax_constant(h->cfg),
      alpha_out_dev ? 1.0 : h->cfg.alpha_relax, h->cfg.slope_relax, L.rface,
      (want_norm && grouped) ? M.qcell : nullptr, (grouped && !alpha_out_dev) ? M.active : nullptr, dWs0, dW0,
      L.color_off[1]);
  if (want_norm && !grouped)
    k_norm_final<DIM + 2><<<1, kBlock, 0, h->stream>>>(M.norm_part, M.norm_blocks, L.n, record ? M.hist : nullptr,
                                                       record ? M.cycle : nullptr, M.max_hist, M.last_norm);
  if (want_norm && grouped) {
    k_group_norm<DIM + 2><<<M.n_groups, kBlock, 0, h->stream>>>(M.qcell, M.goff, M.gidx, record ? M.hist_g : nullptr,
                                                                M.cycle, M.max_hist, M.n_groups, M.last_g);
    if (record) k_bump<<<1, 1, 0, h->stream>>>(M.cycle);
  }
}

// c0_done: the forward step of colour 0 already ran inside the kernel that
// built R and D (fine_residual / coarse_prep with fuse_c0)
template <int DIM, typename T>
// Wcur / Wnext (both null: the level's W, updated in place by a final
// update launch): the state is read from Wcur and the guarded updates are
// written to Wnext by the launches that finalise each colour's increments.
void sweeps(cgks_t* h, MeshDev& M, LevelDev& L, const double* Pf, bool c0_done = false, double* Wcur = nullptr,
            double* Wnext = nullptr) {
  const bool fused = Wnext != nullptr;
  double* W = fused ? Wcur : L.W;
  const double* alpha = h->cfg.df_relax == 1 ? L.alpha : L.relax;
  T* dWs = sizeof(T) == 8 ? (T*)L.dWs64 : (T*)L.dWs32;
  T* dW = sizeof(T) == 8 ? (T*)L.dW64 : (T*)L.dW32;
  const int nc = L.n_colors;
  for (int c = c0_done ? 1 : 0; c < nc - 1; ++c) {
    const int lo = L.color_off[c], hi = L.color_off[c + 1];
    if (hi > lo)
    {
      const int b = fit_block(h, hi - lo, M.blk[B_SWEEP]);
      k_sweep<DIM, T, 0><<<blocks_for(hi - lo, b), b, 0, h->stream>>>(L.topo, lo, hi, W, L.R, Pf, alpha, L.D,
                                                                     L.rface, h->cfg.gamma, dWs, dW);
    }
  }
  if (!(c0_done && nc == 1)) {
    const int lo = L.color_off[nc - 1], hi = L.color_off[nc];
    if (hi > lo)
    {
      const int b = fit_block(h, hi - lo, M.blk[B_SWEEP]);
      k_sweep<DIM, T, 2><<<blocks_for(hi - lo, b), b, 0, h->stream>>>(
          L.topo, lo, hi, W, L.R, Pf, alpha, L.D, L.rface, h->cfg.gamma, dWs, dW, Wnext, M.cnt);
    }
  }
  for (int c = nc - 2; c >= 0; --c) {
    const int lo = L.color_off[c], hi = L.color_off[c + 1];
    if (hi > lo)
    {
      const int b = fit_block(h, hi - lo, M.blk[B_SWEEP]);
      k_sweep<DIM, T, 1><<<blocks_for(hi - lo, b), b, 0, h->stream>>>(
          L.topo, lo, hi, W, L.R, Pf, alpha, L.D, L.rface, h->cfg.gamma, dWs, dW, Wnext, M.cnt);
    }
  }
  const bool fine = &L == &M.lev[0];
  const bool masked = fine && !M.lgrp.empty();
  const int bu = fit_block(h, L.n, M.blk[B_UPDATE]);
  if (fused) {
    // every colour's update was written by its finalising launch, except a
    // single colour's, which the colour-0 forward step finalised
    if (c0_done && nc == 1) {
      CK(cudaMemcpyAsync(Wnext, Wcur, (size_t)L.n * M.nv * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      k_update<DIM, T><<<blocks_for(L.n, bu), bu, 0, h->stream>>>(L.n, h->cfg.gamma, Wnext, dW, M.cnt, nullptr,
                                                                   nullptr);
    }
    return;
  }
  k_update<DIM, T><<<blocks_for(L.n, bu), bu, 0, h->stream>>>(
      L.n, h->cfg.gamma, L.W, dW, M.cnt, masked ? M.lgrp[0] : nullptr, masked ? M.active : nullptr);
}

// TS / fuse_c0: as in fine_residual.  faces_ready: L.Fc and L.rface already
// hold the face fluxes and spectral radii of the current state
template <int DIM, typename TS = double>
void coarse_prep(cgks_t* h, MeshDev& M, LevelDev& L, const double* Pf, bool want_diag, bool fuse_c0 = false,
                 bool faces_ready = false, const double* Wc = nullptr) {
  const PhysParams p = phys(h->cfg, DIM);
  const int bf = fit_block(h, L.faces.nf, M.blk[B_FACE]), bc = fit_block(h, L.n, M.blk[B_CELL]);
  const double* W = Wc ? Wc : L.W;  // the buffer holding the current state
  if (!faces_ready)
    k_face_kfvs<DIM><<<blocks_for(L.faces.nf, bf), bf, 0, h->stream>>>(
        L.faces, W, M.winf, p, L.Fc, want_diag ? L.rface : nullptr);
  const bool fuse = fuse_c0 && want_diag;
  TS* dWs0 = fuse ? (sizeof(TS) == 8 ? (TS*)L.dWs64 : (TS*)L.dWs32) : nullptr;
  TS* dW0 = fuse && L.n_colors == 1 ? (sizeof(TS) == 8 ? (TS*)L.dW64 : (TS*)L.dW32) : nullptr;
  k_coarse_cell<DIM, TS><<<blocks_for(L.n, bc), bc, 0, h->stream>>>(
      L.topo, W, L.Fc, L.rface, Pf, nullptr, h->cfg.df_relax == 1 ? L.alpha : L.relax, h->cfg.gamma, h->cfg.cfl_exp,
      h->cfg.cfl_imp, L.R, want_diag ? L.D : nullptr, dWs0, dW0, L.color_off[1]);
}

// One smoothing step of a two-colour coarse level of at most
// cfg.coarse_cluster_max_cells cells: the face fluxes (unless faces_ready),
// then k_coarse_step_cluster in one thread-block cluster.  Returns false,
// launching nothing, where the level does not qualify.
template <int DIM, typename T>
bool coarse_step_cluster(cgks_t* h, MeshDev& M, LevelDev& L, bool faces_ready, double* Wcur, double* Wnext) {
  const int cs = h->cluster_cs[sizeof(T) == 8 ? 0 : 1];
  if (DIM != 2 || cs < 1 || L.n_colors != 2 || L.n > h->cfg.coarse_cluster_max_cells || L.n < 1) return false;
  const PhysParams p = phys(h->cfg, DIM);
  if (!faces_ready) {
    const int bf = fit_block(h, L.faces.nf, M.blk[B_FACE]);
    k_face_kfvs<DIM><<<blocks_for(L.faces.nf, bf), bf, 0, h->stream>>>(L.faces, Wcur, M.winf, p, L.Fc, L.rface);
    CK(cudaGetLastError());
  }
  T* dWs = sizeof(T) == 8 ? (T*)L.dWs64 : (T*)L.dWs32;
  T* dW = sizeof(T) == 8 ? (T*)L.dW64 : (T*)L.dW32;
  const double* alpha = h->cfg.df_relax == 1 ? L.alpha : L.relax;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3(cs, 1, 1);
  lc.blockDim = dim3(kClusterBlock, 1, 1);
  lc.dynamicSmemBytes = 0;
  lc.stream = h->stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = cs;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  CK(cudaLaunchKernelEx(&lc, k_coarse_step_cluster<DIM, T>, L.topo, (const double*)Wcur, (const double*)L.Fc,
                        (const double*)L.rface, (const double*)L.P, alpha, h->cfg.gamma, h->cfg.cfl_exp,
                        h->cfg.cfl_imp, L.R, L.D, dWs, dW, L.color_off[1], Wnext, M.cnt));
  return true;
}

// blocks per cluster that the coarse-step cluster kernel can run with (16 where
// the device allows that non-portable size, else 8; 0 if neither)
template <typename T>
int coarse_cluster_size() {
  auto kern = k_coarse_step_cluster<2, T>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
    (void)cudaGetLastError();
  }
  for (int cs : {16, 8}) {
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cs, 1, 1);
    lc.blockDim = dim3(kClusterBlock, 1, 1);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = cs;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, kern, &lc) == cudaSuccess && nc >= 1) return cs;
    (void)cudaGetLastError();
  }
  return 0;
}

// FAS forcing P = R* - R(W0) on a coarse level.  The restriction sets W = W0,
// so the face fluxes and spectral radii computed here also serve the first
// smoothing step (coarse_prep with faces_ready).
template <int DIM>
void coarse_forcing(cgks_t* h, MeshDev& M, LevelDev& L) {
  const PhysParams p = phys(h->cfg, DIM);
  const int bf = fit_block(h, L.faces.nf, M.blk[B_FACE]), bc = fit_block(h, L.n, M.blk[B_CELL]);
  k_face_kfvs<DIM><<<blocks_for(L.faces.nf, bf), bf, 0, h->stream>>>(L.faces, L.W0, M.winf, p, L.Fc, L.rface);
  k_coarse_cell<DIM, double><<<blocks_for(L.n, bc), bc, 0, h->stream>>>(L.topo, L.W0, L.Fc, nullptr, nullptr, L.Rstar,
                                                                 L.alpha, h->cfg.gamma, 0.0, 0.0, L.P, nullptr,
                                                                 nullptr, nullptr, 0);
}

// steps 1-3 of the V-cycle: residual + slope update, fine smoothing, residual
template <int DIM, typename T>
void vcycle_pre(cgks_t* h, MeshDev& M) {
  LevelDev& L0 = M.lev[0];
  // 1. residual, norms, slope update with DF, LU-SGS diagonal (and the
  //    forward LU-SGS step of colour 0, fused into the same kernel)
  const bool lusgs = h->cfg.fine_smoother != 1;
  fine_residual<DIM, T>(h, M, true, true, true, true, nullptr, nullptr, lusgs);
  // 2. pre-smoothing: one DF-relaxed LU-SGS step on -R, or the explicit update
  if (!lusgs)
    k_explicit<DIM><<<blocks_for(L0.n), kBlock, 0, h->stream>>>(
        L0.n, h->cfg.gamma, L0.R, L0.dte, L0.vol, L0.W, M.cnt, M.lgrp.empty() ? nullptr : M.lgrp[0],
        M.lgrp.empty() ? nullptr : M.active);
  else
    sweeps<DIM, T>(h, M, L0, nullptr, true);
  if (M.nlev == 1) return;
  // 3. residual at the smoothed state (no slope update); its DF is kept
  fine_residual<DIM>(h, M, false, false, false, false, nullptr, nullptr);
}

// steps 4-8: restriction, forcing, coarse smoothing, prolongation
template <int DIM, typename T>
void vcycle_coarse(cgks_t* h, MeshDev& M) {
  if (M.nlev == 1) return;
  for (int l = 1; l < M.nlev; ++l) {
    LevelDev& F = M.lev[l - 1];
    LevelDev& C = M.lev[l];
    const int br = fit_block(h, C.n, kBlock);
    k_restrict<DIM><<<blocks_for(C.n, br), br, 0, h->stream>>>(C.n, C.ch_off, C.ch_idx, F.vol, C.vol, F.W, F.alpha,
                                                                F.R, C.W0, C.W, C.alpha, C.Rstar);
    coarse_forcing<DIM>(h, M, C);
    // the smoothing steps alternate the state between C.W and C.Wb (each
    // colour's update is written by the launch that finalises it); after an
    // odd number of steps the state is copied back to C.W
    const int nsw = h->cfg.n_sweep_coarse;
    for (int s = 0; s < nsw; ++s) {
      double* Wcur = (s & 1) ? C.Wb : C.W;
      double* Wnext = (s & 1) ? C.W : C.Wb;
      if (!coarse_step_cluster<DIM, T>(h, M, C, s == 0, Wcur, Wnext)) {
        coarse_prep<DIM, T>(h, M, C, C.P, true, true, s == 0, Wcur);
        sweeps<DIM, T>(h, M, C, nullptr, true, Wcur, Wnext);
      }
    }
    if (nsw & 1) CK(cudaMemcpyAsync(C.W, C.Wb, (size_t)C.n * M.nv * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    if (l + 1 < M.nlev) coarse_prep<DIM>(h, M, C, C.P, false);  // R~ = R(W) + P to restrict
  }
  for (int l = M.nlev - 1; l >= 1; --l) {
    LevelDev& F = M.lev[l - 1];
    LevelDev& C = M.lev[l];
    const bool masked = l == 1 && !M.lgrp.empty();
    const int bp = fit_block(h, F.n, kBlock);
    k_prolong<DIM><<<blocks_for(F.n, bp), bp, 0, h->stream>>>(F.n, F.parent, h->cfg.df_prolong ? F.alpha : F.ones,
                                                               C.W, C.W0, h->cfg.gamma, F.W, M.cnt,
                                                               masked ? M.lgrp[0] : nullptr,
                                                               masked ? M.active : nullptr);
  }
}

template <int DIM, typename T>
void vcycle_body(cgks_t* h, MeshDev& M) {
  vcycle_pre<DIM, T>(h, M);
  vcycle_coarse<DIM, T>(h, M);
}

void enqueue_kind(cgks_t* h, MeshDev& M, int kind, int prec);
void ensure_learned(cgks_t* h, MeshDev& M);

cudaGraphExec_t get_graph_kind(cgks_t* h, MeshDev& M, int kind, int prec) {
  if (M.graph[kind][prec]) return M.graph[kind][prec];
  if (kind > 0) ensure_learned(h, M);  // allocations are not allowed during capture
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  try {
    enqueue_kind(h, M, kind, prec);
  } catch (...) {
    cudaStreamEndCapture(h->stream, &g);
    if (g) cudaGraphDestroy(g);
    throw;
  }
  CK(cudaStreamEndCapture(h->stream, &g));
  size_t nn = 0;
  CK(cudaGraphGetNodes(g, nullptr, &nn));
  std::vector<cudaGraphNode_t> nodes(nn);
  if (nn) CK(cudaGraphGetNodes(g, nodes.data(), &nn));
  int nk = 0;
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    CK(cudaGraphNodeGetType(nd, &t));
    nk += t == cudaGraphNodeTypeKernel;
  }
  M.graph_kernels[kind][prec] = nk;
  cudaGraphExec_t ge;
  cudaError_t e = cudaGraphInstantiate(&ge, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  M.graph[kind][prec] = ge;
  return ge;
}

cudaGraphExec_t get_graph(cgks_t* h, MeshDev& M, int mode) { return get_graph_kind(h, M, 0, mode); }

// ---- I/O with permutation ------------------------------------------------
// copy caller rows (original order) into dst (device colour order)
void load_rows(cgks_t* h, MeshDev& M, const LevelDev& L, int w, const double* src, bool on_device, double* dst) {
  const size_t bytes = (size_t)L.n * w * sizeof(double);
  if ((size_t)L.n * w > M.stage_elems) throw ArgError("staging buffer too small");
  if (on_device) CK(cudaMemcpyAsync(M.stage, src, bytes, cudaMemcpyDeviceToDevice, h->stream));
  else CK(cudaMemcpyAsync(M.stage, src, bytes, cudaMemcpyHostToDevice, h->stream));
  k_gather_rows<<<blocks_for((int64_t)L.n * w), kBlock, 0, h->stream>>>(L.n, w, L.iperm, M.stage, dst);
  CK(cudaGetLastError());
  if (!on_device) CK(cudaStreamSynchronize(h->stream));  // host source must outlive the copy
}
void store_rows(cgks_t* h, MeshDev& M, const LevelDev& L, int w, const double* src, bool on_device, double* dst) {
  const size_t bytes = (size_t)L.n * w * sizeof(double);
  if ((size_t)L.n * w > M.stage_elems) throw ArgError("staging buffer too small");
  k_scatter_rows<<<blocks_for((int64_t)L.n * w), kBlock, 0, h->stream>>>(L.n, w, L.iperm, src, M.stage);
  CK(cudaGetLastError());
  if (on_device) CK(cudaMemcpyAsync(dst, M.stage, bytes, cudaMemcpyDeviceToDevice, h->stream));
  else {
    CK(cudaMemcpyAsync(dst, M.stage, bytes, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
  }
}

void require_ready(MeshDev& M, bool state) {
  if (!M.has_hierarchy) throw StateError("cgks_upload_hierarchy has not been called for this mesh");
  if (state && !M.has_state) throw StateError("cgks_init_state has not been called for this mesh");
  if (state && M.winf_h.empty()) throw StateError("cgks_set_freestream has not been called for this mesh");
}

int fail(cgks_t* h, int code, const std::string& msg) {
  if (h) h->err = msg;
  return code;
}

template <class F>
int guarded(cgks_t* h, F&& f) {
  if (!h) return CGKS_ERR_ARG;
  try {
    h->err.clear();
    return f();
  } catch (const ArgError& e) {
    return fail(h, CGKS_ERR_ARG, e.what());
  } catch (const StateError& e) {
    return fail(h, CGKS_ERR_STATE, e.what());
  } catch (const TimeoutError& e) {
    return fail(h, CGKS_ERR_TIMEOUT, e.what());
  } catch (const CudaError& e) {
    return fail(h, CGKS_ERR_CUDA, e.what());
  } catch (const std::bad_alloc&) {
    return fail(h, CGKS_ERR_CUDA, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(h, CGKS_ERR_MESH, e.what());
  }
}

void enqueue_kind(cgks_t* h, MeshDev& M, int kind, int prec);

// after a synchronisation: did a tensor-core network forward give up waiting?
void check_tc_error(cgks_t* h) {
  if (!h->mlp.tc_err) return;
  int e = 0;
  CK(cudaMemcpy(&e, h->mlp.tc_err, sizeof(int), cudaMemcpyDeviceToHost));
  if (e) {
    CK(cudaMemset(h->mlp.tc_err, 0, sizeof(int)));
    throw TimeoutError("the tensor-core network forward gave up waiting for its MMAs");
  }
}

// learned V-cycles with the fallback policy (host-side state machine)
int run_learned(cgks_t* h, MeshDev& M, int n_cycles, double* norms_out, int* cycles_done) {
  const int nv = M.nv;
  cudaGraphExec_t gp = get_graph_kind(h, M, 0, CGKS_MIXED);
  cudaGraphExec_t gl = get_graph_kind(h, M, 1, CGKS_MIXED);
  cudaGraphExec_t gj = get_graph_kind(h, M, 2, CGKS_MIXED);
  int start = 0;
  CK(cudaMemcpyAsync(&start, M.cycle, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  for (double& x : M.lstats) x = 0;
  for (int i = 5; i < 10; ++i) M.lstats[i] = -1;
  bool disabled = false;
  int fallback = 0, done = 0, status = CGKS_OK;
  std::vector<double> rho;      // RMS density residual per cycle
  std::vector<char> learned;    // whether the cycle applied the network
  double ref = -1.0;
  for (int k = 0; k < n_cycles; ++k) {
    const int je_every = h->cfg.learned_judge_every;
    const bool judge = !disabled && fallback == 0 && je_every > 0 && k % je_every == 0;  // cycles 0, J, 2J, ...
    const bool use_net = !disabled && fallback == 0 && !judge;
    CK(cudaGraphLaunch(judge ? gj : (use_net ? gl : gp), h->stream));
    double r = 0.0, je[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const int idx = start + k;
    if (idx < M.max_hist)
      CK(cudaMemcpyAsync(&r, M.hist + (size_t)idx * 2 * nv, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (judge) CK(cudaMemcpyAsync(je, M.judge_out, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    done++;
    rho.push_back(r);
    learned.push_back(use_net);
    if (ref < 0) ref = r;
    M.lstats[use_net ? 0 : 1] += 1;
    if (judge) {
      M.lstats[2] += 1;
      const double e = je[0] + je[1] + je[2] + je[3], t = je[4] + je[5] + je[6] + je[7];
      const double err = t > 0 ? std::sqrt(e / t) : 0.0;
      M.lstats[5] = err;
      for (int v = 0; v < 4; ++v) M.lstats[6 + v] = je[4 + v] > 0 ? std::sqrt(je[v] / je[4 + v]) : 0.0;
      if (err > h->cfg.learned_max_error) disabled = true;
    }
    if (fallback > 0) fallback--;
    // stall: the last five cycles all learned and less than 1 % drop, or 1.5x growth
    const int n = (int)rho.size();
    if (use_net && n >= 2 && rho[n - 1] > 1.5 * rho[n - 2]) {
      fallback = 10;
      M.lstats[3] += 1;
    } else if (use_net && n >= 6) {
      bool all = true;
      for (int i = n - 5; i < n; ++i) all = all && learned[i];
      if (all && rho[n - 1] > 0.99 * rho[n - 6]) {
        fallback = 10;
        M.lstats[3] += 1;
      }
    }
    if (!std::isfinite(r) || (ref > 0 && r > h->cfg.diverge_factor * ref)) {
      status = CGKS_ERR_DIVERGED;
      break;
    }
    if (ref > 0 && r <= h->cfg.tol * ref) break;
  }
  M.lstats[4] = disabled ? 1 : 0;
  if (norms_out) {
    std::vector<double> hist((size_t)done * 2 * nv);
    if (done)
      CK(cudaMemcpy(hist.data(), M.hist + (size_t)start * 2 * nv, hist.size() * sizeof(double),
                    cudaMemcpyDeviceToHost));
    for (int i = 0; i < n_cycles; ++i)
      for (int j = 0; j < 2 * nv; ++j)
        norms_out[(size_t)i * 2 * nv + j] = i < done ? hist[(size_t)i * 2 * nv + j] : -1.0;
  }
  if (cycles_done) *cycles_done = done;
  check_tc_error(h);
  return status;
}

}  // namespace
}  // namespace cgks

using namespace cgks;

extern "C" {

int cgks_default_config(cgks_config* c) {
  if (!c) return CGKS_ERR_ARG;
  c->gamma = 1.4;
  c->cfl_imp = 10.0;
  c->cfl_exp = 0.5;
  c->tau_c1 = 0.01;
  c->tau_c2 = 1.0;
  c->weno_gamma_high = 0.95;
  c->weno_eps = 1e-15;
  c->r_safety = 1.0;
  c->n_sweep_coarse = 6;
  c->n_pre = 1;
  c->n_post = 0;
  c->check_every = 10;
  c->tol = 1e-10;
  c->diverge_factor = 1e6;
  c->fine_smoother = 0;
  c->df_relax = 1;
  c->df_prolong = 1;
  c->df_gate = 0.9;
  c->learned_judge_every = 20;
  c->learned_max_error = 0.5;
  c->flux_precision = 0;
  c->relax_beta = 0.5;
  c->mu = 0.0;
  c->slope_relax = 1.0;
  c->alpha_relax = 1.0;
  c->learned_scale = 0;
  c->coarse_cluster_max_cells = 0;
  return CGKS_OK;
}

int cgks_create(cgks_t** out, const cgks_config* cfg, void* stream) {
  if (!out) return CGKS_ERR_ARG;
  *out = nullptr;
  cgks_t* h = new (std::nothrow) cgks_ctx();
  if (!h) return CGKS_ERR_CUDA;
  h->err.reserve(512);  // error messages of the no-allocation entry point fit without reallocating
  if (cfg) h->cfg = *cfg;
  else cgks_default_config(&h->cfg);
  if (h->cfg.n_pre != 1 || h->cfg.n_post != 0 || h->cfg.n_sweep_coarse < 1 || !(h->cfg.gamma > 1.0) ||
      h->cfg.r_safety != 1.0 || !(h->cfg.weno_gamma_high > 0.0 && h->cfg.weno_gamma_high <= 1.0) ||
      h->cfg.check_every < 1 || (h->cfg.fine_smoother != 0 && h->cfg.fine_smoother != 1) ||
      (h->cfg.flux_precision != 0 && h->cfg.flux_precision != 1) ||
      (h->cfg.df_relax < 0 || h->cfg.df_relax > 2) || (h->cfg.df_prolong != 0 && h->cfg.df_prolong != 1) ||
      !(h->cfg.relax_beta >= 0.0 && h->cfg.relax_beta <= 1.0) || !(h->cfg.mu >= 0.0 && h->cfg.mu < 1e300) ||
      !(h->cfg.tau_c1 > 0.0 && h->cfg.tau_c1 < 1e300) || !(h->cfg.tau_c2 >= 0.0 && h->cfg.tau_c2 < 1e300) ||
      !(h->cfg.cfl_imp > 0.0 && h->cfg.cfl_imp < 1e300) || !(h->cfg.cfl_exp > 0.0 && h->cfg.cfl_exp < 1e300) ||
      !(h->cfg.weno_eps > 0.0 && h->cfg.weno_eps < 1e300) ||
      !(h->cfg.slope_relax > 0.0 && h->cfg.slope_relax <= 1.0) ||
      !(h->cfg.alpha_relax > 0.0 && h->cfg.alpha_relax <= 1.0) ||
      (h->cfg.learned_scale != 0 && h->cfg.learned_scale != 1) || h->cfg.coarse_cluster_max_cells < 0) {
    delete h;
    return CGKS_ERR_ARG;
  }
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) {
      h->device = dev;
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
        h->sms = sms;
      // the coarse-step cluster kernel's cluster size on this device
      h->cluster_cs[0] = cgks::coarse_cluster_size<double>();
      h->cluster_cs[1] = cgks::coarse_cluster_size<float>();
    }
  }
  if (stream) {
    h->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete h;
      return CGKS_ERR_CUDA;
    }
    h->own_stream = true;
  }
  *out = h;
  return CGKS_OK;
}

int cgks_destroy(cgks_t* h) {
  if (!h) return CGKS_OK;
  cudaStreamSynchronize(h->stream);
  h->meshes.clear();
  h->scratch.clear();
  if (h->pin) cudaFreeHost(h->pin);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return CGKS_OK;
}

const char* cgks_last_error(cgks_t* h) { return h ? h->err.c_str() : "null handle"; }

int cgks_synchronize(cgks_t* h) {
  return guarded(h, [&]() -> int {
    CK(cudaStreamSynchronize(h->stream));
    check_tc_error(h);
    return CGKS_OK;
  });
}

int cgks_upload_mesh(cgks_t* h, int mesh_id, int dim, int64_t n_cells, const int32_t* cell_nodes,
                     const double* cell_xyz, int64_t n_bfaces, const int32_t* bface_nodes,
                     const int32_t* bface_tag) {
  return guarded(h, [&]() -> int {
    if ((dim != 2 && dim != 3) || n_cells <= 0 || !cell_nodes || !cell_xyz || n_bfaces < 0 ||
        (n_bfaces > 0 && (!bface_nodes || !bface_tag)) || n_cells >= (1ll << 30))
      throw ArgError("invalid mesh arguments");
    for (int64_t b = 0; b < n_bfaces; ++b)
      if (bface_tag[b] < CGKS_TAG_WALL || bface_tag[b] > CGKS_TAG_FARFIELD_RIEMANN) throw ArgError("unknown boundary tag");
    auto M = std::make_unique<MeshDev>();
    M->dim = dim;
    M->nv = dim + 2;
    try {
      build_fine_level(dim, n_cells, cell_nodes, cell_xyz, n_bfaces, bface_nodes, bface_tag, M->H.fine);
    } catch (const std::runtime_error& e) {
      return fail(h, CGKS_ERR_MESH, e.what());
    }
    CK(cudaStreamSynchronize(h->stream));
    h->meshes[mesh_id] = std::move(M);
    return CGKS_OK;
  });
}

int cgks_upload_mesh_mixed(cgks_t* h, int mesh_id, int64_t n_cells, const int32_t* cell_type,
                           const int64_t* cell_node_off, const int32_t* cell_nodes, const double* cell_xyz,
                           int64_t n_bfaces, const int64_t* bface_node_off, const int32_t* bface_nodes,
                           const int32_t* bface_tag) {
  return guarded(h, [&]() -> int {
    if (n_cells <= 0 || n_cells >= (1ll << 30) || !cell_type || !cell_node_off || !cell_nodes || !cell_xyz ||
        n_bfaces < 0 || (n_bfaces > 0 && (!bface_node_off || !bface_nodes || !bface_tag)))
      throw ArgError("invalid mesh arguments");
    if (h->cfg.flux_precision != 0) throw ArgError("mixed-element meshes take the FP64 flux (flux_precision 0)");
    for (int64_t b = 0; b < n_bfaces; ++b)
      if (bface_tag[b] < CGKS_TAG_WALL || bface_tag[b] > CGKS_TAG_FARFIELD_RIEMANN) throw ArgError("unknown boundary tag");
    auto M = std::make_unique<MeshDev>();
    M->dim = 3;
    M->nv = 5;
    try {
      build_fine_level_mixed(n_cells, cell_type, cell_node_off, cell_nodes, cell_xyz, n_bfaces, bface_node_off,
                             bface_nodes, bface_tag, M->H.fine);
    } catch (const std::runtime_error& e) {
      return fail(h, CGKS_ERR_MESH, e.what());
    }
    CK(cudaStreamSynchronize(h->stream));
    h->meshes[mesh_id] = std::move(M);
    return CGKS_OK;
  });
}

int cgks_upload_hierarchy(cgks_t* h, int mesh_id, int n_levels, const int32_t* const* parent) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    if (n_levels < 1 || n_levels > 8 || (n_levels > 1 && !parent)) throw ArgError("invalid level count");
    M.H.coarse.clear();
    M.drop_graphs();
    try {
      for (int l = 1; l < n_levels; ++l) {
        if (!parent[l - 1]) throw ArgError("null parent array");
        CoarseLevel C;
        build_coarse_level(M.H, l - 1, parent[l - 1], C);
        M.H.coarse.push_back(std::move(C));
      }
    } catch (const ArgError&) {
      throw;
    } catch (const std::runtime_error& e) {
      return fail(h, CGKS_ERR_MESH, e.what());
    }
    CK(cudaStreamSynchronize(h->stream));
    M.lgrp.clear();
    M.gpool.clear();
    M.qcell = nullptr;
    M.n_groups = 1;
    if (M.winf_h.size() > (size_t)M.nv) M.winf_h.resize(M.nv);
    M.pool.clear();
    M.nlev = n_levels;
    build_fine_device(M);
    build_levels_device(M, h->cfg);
    M.has_hierarchy = true;
    M.has_state = false;
    CK(cudaDeviceSynchronize());
    return CGKS_OK;
  });
}

int cgks_agglomerate(cgks_t* h, int dim, int64_t n_cells, const int32_t* cell_nodes, const double* cell_xyz,
                     int64_t n_bfaces, const int32_t* bface_nodes, const int32_t* bface_tag, int n_levels,
                     int passes, double min_skew, int32_t* parents, int64_t* level_cells) {
  return guarded(h, [&]() -> int {
    if ((dim != 2 && dim != 3) || n_cells <= 0 || !cell_nodes || !cell_xyz || n_bfaces < 0 ||
        (n_bfaces > 0 && (!bface_nodes || !bface_tag)) || n_cells >= (1ll << 30) || n_levels < 1 ||
        n_levels > 8 || passes < 1 || passes > 8 || !(min_skew >= -1.0 && min_skew < 1.0) || !level_cells ||
        (n_levels > 1 && !parents))
      throw ArgError("invalid agglomeration arguments");
    std::vector<std::vector<int32_t>> P;
    try {
      agglomerate(dim, n_cells, cell_nodes, cell_xyz, n_bfaces, bface_nodes, bface_tag, n_levels, passes,
                  min_skew, P);
    } catch (const std::runtime_error& e) {
      return fail(h, CGKS_ERR_MESH, e.what());
    }
    level_cells[0] = n_cells;
    for (int l = 1; l < n_levels; ++l) {
      const std::vector<int32_t>& p = P[l - 1];
      std::memcpy(parents + (size_t)(l - 1) * n_cells, p.data(), p.size() * sizeof(int32_t));
      level_cells[l] = 1 + *std::max_element(p.begin(), p.end());
    }
    return CGKS_OK;
  });
}

int cgks_mesh_info(cgks_t* h, int mesh_id, int* n_levels, int64_t* out) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    const int nl = 1 + (int)M.H.coarse.size();
    if (n_levels) *n_levels = nl;
    if (out) {
      out[0] = M.H.fine.n;
      out[1] = M.H.fine.n_colors;
      out[2] = M.H.fine.nf;
      out[3] = M.H.fine.nf - M.H.fine.nf_int;
      for (int l = 1; l < nl; ++l) {
        const CoarseLevel& C = M.H.coarse[l - 1];
        int64_t nb = 0;
        for (int64_t f = 0; f < C.nf; ++f) nb += C.fR[f] < 0;
        out[4 * l + 0] = C.n;
        out[4 * l + 1] = C.n_colors;
        out[4 * l + 2] = C.nf;
        out[4 * l + 3] = nb;
      }
    }
    return CGKS_OK;
  });
}

int cgks_get_coloring(cgks_t* h, int mesh_id, int level, int32_t* colors) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    if (!colors || level < 0 || level > (int)M.H.coarse.size()) throw ArgError("invalid level");
    const std::vector<int32_t>& c = level == 0 ? M.H.fine.color_orig : M.H.coarse[level - 1].color_orig;
    std::memcpy(colors, c.data(), c.size() * sizeof(int32_t));
    return CGKS_OK;
  });
}

int cgks_get_hierarchy(cgks_t* h, int mesh_id, int level, int32_t* order, int32_t* parent) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    if (level < 0 || level > (int)M.H.coarse.size()) throw ArgError("invalid level");
    if (parent && level == (int)M.H.coarse.size()) throw ArgError("the coarsest level has no parent map");
    const std::vector<int64_t>& ip = level == 0 ? M.H.fine.iperm : M.H.coarse[level - 1].iperm;
    if (order)
      for (size_t i = 0; i < ip.size(); ++i) order[i] = (int32_t)ip[i];
    if (parent) {
      // parent_of_fine: this level's new ids -> next level's new ids; map both to original ids
      const CoarseLevel& C = M.H.coarse[level];
      for (size_t i = 0; i < ip.size(); ++i) parent[ip[i]] = (int32_t)C.iperm[C.parent_of_fine[i]];
    }
    return CGKS_OK;
  });
}

int cgks_set_freestream(cgks_t* h, int mesh_id, const double* w) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    if (!w) throw ArgError("null free stream");
    M.winf_h.assign(w, w + M.nv);
    if (M.winf) CK(cudaMemcpyAsync(M.winf, M.winf_h.data(), M.nv * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_set_state(cgks_t* h, int mesh_id, const double* W, const double* grad, const double* alpha,
                   int on_device) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, false);
    LevelDev& L = M.lev[0];
    if (W) load_rows(h, M, L, M.nv, W, on_device, L.W);
    if (grad) load_rows(h, M, L, M.nv * M.dim, grad, on_device, M.G);
    if (alpha) load_rows(h, M, L, 1, alpha, on_device, L.alpha);
    if (W) M.has_state = true;
    return CGKS_OK;
  });
}

int cgks_init_state(cgks_t* h, int mesh_id, const double* W, const double* grad, int on_device) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, false);
    if (!W) throw ArgError("null state");
    LevelDev& L = M.lev[0];
    load_rows(h, M, L, M.nv, W, on_device, L.W);
    if (grad) load_rows(h, M, L, M.nv * M.dim, grad, on_device, M.G);
    else CK(cudaMemsetAsync(M.G, 0, (size_t)L.n * M.nv * M.dim * sizeof(double), h->stream));
    k_fill<<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.n, 1.0, L.alpha);
    CK(cudaMemsetAsync(M.cnt, 0, sizeof(Counters), h->stream));
    CK(cudaMemsetAsync(M.cycle, 0, sizeof(int), h->stream));
    CK(cudaStreamSynchronize(h->stream));
    M.has_state = true;
    return CGKS_OK;
  });
}

int cgks_get_state(cgks_t* h, int mesh_id, double* W, double* grad, double* alpha, int on_device) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    LevelDev& L = M.lev[0];
    if (W) store_rows(h, M, L, M.nv, L.W, on_device, W);
    if (grad) store_rows(h, M, L, M.nv * M.dim, M.G, on_device, grad);
    if (alpha) store_rows(h, M, L, 1, L.alpha, on_device, alpha);
    return CGKS_OK;
  });
}

int cgks_residual(cgks_t* h, int mesh_id, int level, const double* W_in, double* R_out, double* grad_new_out,
                  double* alpha_out, int on_device) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    if (level < 0 || level >= M.nlev) throw ArgError("invalid level");
    if (level == 0) {
      require_ready(M, true);
      LevelDev& L = M.lev[0];
      // alpha of the state is the previous DF; write the new one to a scratch row
      double* anew = L.D;  // D is rebuilt before every sweep, so it can hold the new DF here
      if (M.dim == 2) fine_residual<2>(h, M, false, false, true, false, anew, M.gradnew);
      else fine_residual<3>(h, M, false, false, true, false, anew, M.gradnew);
      CK(cudaGetLastError());
      if (R_out) store_rows(h, M, L, M.nv, L.R, on_device, R_out);
      if (grad_new_out) store_rows(h, M, L, M.nv * M.dim, M.gradnew, on_device, grad_new_out);
      if (alpha_out) store_rows(h, M, L, 1, anew, on_device, alpha_out);
      return CGKS_OK;
    }
    require_ready(M, false);
    if (!W_in || grad_new_out || alpha_out) throw ArgError("coarse residual takes W_in and returns R only");
    if (M.winf_h.empty()) throw StateError("cgks_set_freestream has not been called for this mesh");
    LevelDev& L = M.lev[level];
    load_rows(h, M, L, M.nv, W_in, on_device, L.W0);
    const PhysParams p = phys(h->cfg, M.dim);
    // R(W) of the level's faces with zero forcing
    if (M.dim == 2) {
      k_face_kfvs<2><<<blocks_for(L.faces.nf), kBlock, 0, h->stream>>>(L.faces, L.W0, M.winf, p, L.Fc, nullptr);
      k_coarse_cell<2, double><<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.topo, L.W0, L.Fc, nullptr, nullptr, nullptr, L.alpha, h->cfg.gamma, 0.0, 0.0, L.Rstar, nullptr, nullptr, nullptr, 0);
    } else {
      k_face_kfvs<3><<<blocks_for(L.faces.nf), kBlock, 0, h->stream>>>(L.faces, L.W0, M.winf, p, L.Fc, nullptr);
      k_coarse_cell<3, double><<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.topo, L.W0, L.Fc, nullptr, nullptr, nullptr, L.alpha, h->cfg.gamma, 0.0, 0.0, L.Rstar, nullptr, nullptr, nullptr, 0);
    }
    CK(cudaGetLastError());
    if (R_out) store_rows(h, M, L, M.nv, L.Rstar, on_device, R_out);
    return CGKS_OK;
  });
}

int cgks_reconstruct(cgks_t* h, int mesh_id, double* coef_out, double* dt_exp_out, double* dt_imp_out,
                     int on_device) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    LevelDev& L = M.lev[0];
    if (M.dim == 2) launch_recon<2>(h, M);
    else launch_recon<3>(h, M);
    CK(cudaGetLastError());
    const int nc = M.dim == 2 ? 6 : 10;
    if (coef_out) store_rows(h, M, L, M.nv * nc, M.coef, on_device, coef_out);
    if (dt_exp_out) store_rows(h, M, L, 1, L.dte, on_device, dt_exp_out);
    if (dt_imp_out) store_rows(h, M, L, 1, L.dti, on_device, dt_imp_out);
    return CGKS_OK;
  });
}

int cgks_lusgs(cgks_t* h, int mesh_id, int level, int mode, double* W_inout, const double* rhs,
               const double* alpha, const double* dt_exp, const double* dt_imp, double* dW_out, int on_device) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, false);
    if (level < 0 || level >= M.nlev || !W_inout || !rhs || !alpha || !dt_exp || !dt_imp ||
        (mode != CGKS_PLAIN_FP64 && mode != CGKS_MIXED))
      throw ArgError("invalid LU-SGS arguments");
    if (M.winf_h.empty()) throw StateError("cgks_set_freestream has not been called for this mesh");
    LevelDev& L = M.lev[level];
    const int nv = M.nv;
    const size_t wb = (size_t)L.n * nv * sizeof(double);
    // the level's buffers are used; the fine state (W, alpha) is saved and restored
    if (level == 0) {
      CK(cudaMemcpyAsync(L.W0, L.W, wb, cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(L.Rstar, L.alpha, L.n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    load_rows(h, M, L, nv, W_inout, on_device, L.W);
    load_rows(h, M, L, nv, rhs, on_device, L.R);
    load_rows(h, M, L, 1, alpha, on_device, L.alpha);
    load_rows(h, M, L, 1, dt_exp, on_device, L.dte);
    load_rows(h, M, L, 1, dt_imp, on_device, L.dti);
    k_scale<<<blocks_for((int64_t)L.n * nv), kBlock, 0, h->stream>>>((int64_t)L.n * nv, -1.0, L.R);  // kernels take R = -rhs
    const PhysParams pp = phys(h->cfg, M.dim);
    if (M.dim == 2) {
      k_face_kfvs<2><<<blocks_for(L.faces.nf), kBlock, 0, h->stream>>>(L.faces, L.W, M.winf, pp, nullptr, L.rface);
      k_diag<2><<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.topo, L.rface, L.alpha, L.dte, L.dti, L.D);
      if (mode == CGKS_MIXED) sweeps<2, float>(h, M, L, nullptr);
      else sweeps<2, double>(h, M, L, nullptr);
    } else {
      k_face_kfvs<3><<<blocks_for(L.faces.nf), kBlock, 0, h->stream>>>(L.faces, L.W, M.winf, pp, nullptr, L.rface);
      k_diag<3><<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.topo, L.rface, L.alpha, L.dte, L.dti, L.D);
      if (mode == CGKS_MIXED) sweeps<3, float>(h, M, L, nullptr);
      else sweeps<3, double>(h, M, L, nullptr);
    }
    CK(cudaGetLastError());
    store_rows(h, M, L, nv, L.W, on_device, W_inout);
    if (dW_out) {
      const double* src = L.dW64;
      if (mode == CGKS_MIXED) {
        k_f2d<<<blocks_for((int64_t)L.n * nv), kBlock, 0, h->stream>>>((int64_t)L.n * nv, L.dW32, L.P);
        src = L.P;
      }
      store_rows(h, M, L, nv, src, on_device, dW_out);
    }
    if (level == 0) {
      CK(cudaMemcpyAsync(L.W, L.W0, wb, cudaMemcpyDeviceToDevice, h->stream));
      CK(cudaMemcpyAsync(L.alpha, L.Rstar, L.n * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_smooth(cgks_t* h, int mesh_id, int level, int n_sweeps) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (level != 0 || n_sweeps < 0) throw ArgError("only fine-level smoothing is exposed");
    for (int s = 0; s < n_sweeps; ++s) {
      if (M.dim == 2) {
        fine_residual<2>(h, M, true, true, true, false, nullptr, nullptr);
        sweeps<2, double>(h, M, M.lev[0], nullptr);
      } else {
        fine_residual<3>(h, M, true, true, true, false, nullptr, nullptr);
        sweeps<3, double>(h, M, M.lev[0], nullptr);
      }
    }
    CK(cudaGetLastError());
    return CGKS_OK;
  });
}

int cgks_vcycle(cgks_t* h, const int* mesh_ids, int n_meshes, int n_cycles, int mode, double* norms_out,
                int* cycles_done) {
  return guarded(h, [&]() -> int {
    if (!mesh_ids || n_meshes < 1 || n_cycles < 0 ||
        (mode != CGKS_PLAIN_FP64 && mode != CGKS_MIXED && mode != CGKS_LEARNED))
      throw ArgError("invalid V-cycle arguments");
    int status = CGKS_OK;
    if (mode == CGKS_LEARNED) {
      for (int k = 0; k < n_meshes; ++k) {
        MeshDev& M = get_mesh(h, mesh_ids[k]);
        require_ready(M, true);
        const int rc = run_learned(h, M, n_cycles, norms_out ? norms_out + (size_t)k * n_cycles * 2 * M.nv : nullptr,
                                   cycles_done ? cycles_done + k : nullptr);
        if (rc != CGKS_OK) status = rc;
      }
      if (status != CGKS_OK) h->err = "residual diverged or became non-finite";
      return status;
    }
    for (int k = 0; k < n_meshes; ++k) {
      MeshDev& M = get_mesh(h, mesh_ids[k]);
      require_ready(M, true);
      const int nv2 = 2 * M.nv;
      cudaGraphExec_t g = get_graph(h, M, mode);
      // one pinned read per chunk: the packed history (k_pack_hist) and the counters
      const int cmax = std::max(1, std::min(h->cfg.check_every, n_cycles));
      const size_t pack_n = 3 + (size_t)cmax * nv2;
      const size_t pin_bytes = pack_n * sizeof(double) + sizeof(Counters);
      if (h->pin_cap < pin_bytes) {
        if (h->pin) CK(cudaFreeHost(h->pin));
        h->pin = nullptr;
        h->pin_cap = 0;
        CK(cudaMallocHost(&h->pin, pin_bytes));
        h->pin_cap = pin_bytes;
      }
      if (h->pack.bytes < pack_n * sizeof(double)) h->pack.alloc(pack_n * sizeof(double));
      double* pk = h->pin;
      Counters* pc = reinterpret_cast<Counters*>(h->pin + pack_n);
      int done = 0;
      bool stop = false;
      while (done < n_cycles && !stop) {
        const int chunk = std::min(cmax, n_cycles - done);
        for (int i = 0; i < chunk; ++i) CK(cudaGraphLaunch(g, h->stream));
        k_pack_hist<<<1, 256, 0, h->stream>>>(M.hist, M.cycle, M.max_hist, nv2, chunk, h->pack.as<double>());
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(pk, h->pack.p, (3 + (size_t)chunk * nv2) * sizeof(double), cudaMemcpyDeviceToHost,
                           h->stream));
        CK(cudaMemcpyAsync(pc, M.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        if (norms_out)
          for (int i = 0; i < chunk; ++i)
            for (int j = 0; j < nv2; ++j)
              norms_out[((size_t)k * n_cycles + done + i) * nv2 + j] = pk[3 + (size_t)i * nv2 + j];
        done += chunk;
        if (pk[0] > 0 && M.max_hist > 0) {
          const double first = pk[1], last = pk[2];
          if (!std::isfinite(last) || (first > 0 && last > h->cfg.diverge_factor * first)) {
            status = CGKS_ERR_DIVERGED;
            stop = true;
          } else if (first > 0 && last <= h->cfg.tol * first) {
            stop = true;
          }
        }
      }
      if (done == 0) {
        CK(cudaMemcpyAsync(pc, M.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
      }
      if (pc->nonfinite > 0) status = CGKS_ERR_DIVERGED;
      if (norms_out)
        for (int i = done; i < n_cycles; ++i)
          for (int j = 0; j < nv2; ++j) norms_out[((size_t)k * n_cycles + i) * nv2 + j] = -1.0;
      if (cycles_done) cycles_done[k] = done;
    }
    if (status != CGKS_OK) h->err = "residual diverged or became non-finite";
    return status;
  });
}

int cgks_residual_norms(cgks_t* h, int mesh_id, int level, double* out) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (level != 0 || !out) throw ArgError("fine-level norms only");
    CK(cudaMemcpyAsync(out, M.last_norm, 2 * M.nv * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_counters(cgks_t* h, int mesh_id, uint64_t* out) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, false);
    if (!out) throw ArgError("null output");
    Counters c{};
    CK(cudaMemcpyAsync(&c, M.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    out[0] = c.recon_fallback;
    out[1] = c.update_halved;
    out[2] = c.update_zeroed;
    out[3] = c.nonfinite;
    return CGKS_OK;
  });
}

int cgks_gks_points(cgks_t* h, int dim, int64_t n, const double* Wl, const double* Gl, const double* Wr,
                    const double* Gr, const double* dt, double* F, double* Wt, double* alpha) {
  return guarded(h, [&]() -> int {
    if ((dim != 2 && dim != 3) || n < 0 || n >= (1ll << 31) || !Wl || !Gl || !Wr || !Gr || !dt || !F || !Wt || !alpha)
      throw ArgError("invalid point-flux arguments");
    if (n == 0) return CGKS_OK;
    const PhysParams p = phys(h->cfg, dim);
    if (dim == 2) k_gks_points<2><<<blocks_for(n), kBlock, 0, h->stream>>>((int)n, p, Wl, Gl, Wr, Gr, dt, F, Wt, alpha);
    else k_gks_points<3><<<blocks_for(n), kBlock, 0, h->stream>>>((int)n, p, Wl, Gl, Wr, Gr, dt, F, Wt, alpha);
    CK(cudaGetLastError());
    return CGKS_OK;
  });
}

int cgks_vcycle_launch(cgks_t* h, const int* mesh_ids, int n_meshes, int n_cycles, int mode) {
  return guarded(h, [&]() -> int {
    if (!mesh_ids || n_meshes < 1 || n_cycles < 0 || (mode != CGKS_PLAIN_FP64 && mode != CGKS_MIXED))
      throw ArgError("invalid V-cycle arguments");
    for (int k = 0; k < n_meshes; ++k) {
      MeshDev& M = get_mesh(h, mesh_ids[k]);
      require_ready(M, true);
      cudaGraphExec_t g = get_graph(h, M, mode);
      for (int i = 0; i < n_cycles; ++i) CK(cudaGraphLaunch(g, h->stream));
    }
    return CGKS_OK;
  });
}

int cgks_dword_selftest(cgks_t* h, int64_t n, const double* a, const double* b, double* out) {
  return guarded(h, [&]() -> int {
    if (n < 0 || (n > 0 && (!a || !b || !out))) throw ArgError("invalid self-test arguments");
    if (n == 0) return CGKS_OK;
    DBuf da, db, dout;
    da.alloc((size_t)n * 8);
    db.alloc((size_t)n * 8);
    dout.alloc((size_t)n * 7 * 8);
    CK(cudaMemcpyAsync(da.p, a, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(db.p, b, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream));
    k_dword_selftest<<<blocks_for(n), kBlock, 0, h->stream>>>((int)n, da.as<double>(), db.as<double>(),
                                                              dout.as<double>());
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dout.p, (size_t)n * 7 * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_special_selftest(cgks_t* h, int64_t n, const double* x, double* out) {
  return guarded(h, [&]() -> int {
    if (n < 0 || n >= (1ll << 31) || (n > 0 && (!x || !out))) throw ArgError("invalid self-test arguments");
    if (n == 0) return CGKS_OK;
    DBuf dx, dout;
    dx.alloc((size_t)n * 8);
    dout.alloc((size_t)n * 5 * 8);
    CK(cudaMemcpyAsync(dx.p, x, (size_t)n * 8, cudaMemcpyHostToDevice, h->stream));
    k_special_selftest<<<blocks_for(n), kBlock, 0, h->stream>>>((int)n, dx.as<double>(), dout.as<double>());
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(out, dout.p, (size_t)n * 5 * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_fma_probe(cgks_t* h, int precision, double* tflops) {
  return guarded(h, [&]() -> int {
    if (!tflops || (precision != 0 && precision != 1)) throw ArgError("invalid probe arguments");
    int dev = 0, sms = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int blocks = sms * 16, threads = 256, chains = 8;
    const int iters = precision == 0 ? 4096 : 65536;
    DBuf out;
    out.alloc((size_t)blocks * threads * 8);
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    float ms = 0.f;
    for (int rep = 0; rep < 4; ++rep) {  // the last of 4 runs is timed (warm clocks)
      CK(cudaEventRecord(e0, h->stream));
      if (precision == 0)
        k_fma_probe<double, 8><<<blocks, threads, 0, h->stream>>>(out.as<double>(), iters, 0.999999, 1e-7);
      else
        k_fma_probe<float, 8><<<blocks, threads, 0, h->stream>>>(out.as<float>(), iters, 0.999999f, 1e-7f);
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      CK(cudaEventElapsedTime(&ms, e0, e1));
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *tflops = 2.0 * blocks * threads * (double)iters * chains / (ms * 1e-3) / 1e12;
    return CGKS_OK;
  });
}

int cgks_run_stage(cgks_t* h, int mesh_id, int stage) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (stage < 0 || stage > 2) throw ArgError("stage must be 0, 1 or 2");
    LevelDev& L = M.lev[0];
    if (stage == 0) {
      if (M.dim == 2) launch_recon<2>(h, M);
      else launch_recon<3>(h, M);
    } else if (stage == 1) {
      if (M.dim == 2) launch_flux<2>(h, M);
      else launch_flux<3>(h, M);
    } else {
      if (M.dim == 2)
        k_gather<2><<<blocks_for(L.n), kBlock, 0, h->stream>>>(
            M.fine, L.topo, M.Fface, M.Wface, M.aface, L.W, M.winf, h->cfg.gamma, L.dte, L.dti, L.R, nullptr, L.alpha,
            L.D, nullptr, nullptr, h->cfg.df_relax == 1 ? -1.0 : relax_constant(h->cfg), h->cfg.alpha_relax, 1.0,
            L.rface, nullptr, nullptr);
      else
        (M.H.fine.mixed ? k_gather<3, double, 1> : k_gather<3, double>)<<<blocks_for(L.n), kBlock, 0, h->stream>>>(
            M.fine, L.topo, M.Fface, M.Wface, M.aface, L.W, M.winf, h->cfg.gamma, L.dte, L.dti, L.R, nullptr, L.alpha,
            L.D, nullptr, nullptr, h->cfg.df_relax == 1 ? -1.0 : relax_constant(h->cfg), h->cfg.alpha_relax, 1.0,
            L.rface, nullptr, nullptr, nullptr, nullptr, 0);
    }
    CK(cudaGetLastError());
    return CGKS_OK;
  });
}

int cgks_launch_count(cgks_t* h, int mesh_id, int mode, int* count) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (!count || (mode != CGKS_PLAIN_FP64 && mode != CGKS_MIXED)) throw ArgError("invalid arguments");
    get_graph(h, M, mode);
    *count = M.graph_kernels[0][mode];
    return CGKS_OK;
  });
}

int cgks_set_groups(cgks_t* h, int mesh_id, int n_groups, const int32_t* group_of_cell, const double* winf) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, false);
    if (n_groups < 1 || !group_of_cell || !winf) throw ArgError("invalid group arguments");
    const int nv = M.nv;
    const FineLevel& F = M.H.fine;
    // group of every cell on every level (new ids); coarse cells inherit the
    // group of their children, which must agree
    std::vector<std::vector<int>> grp(M.nlev);
    grp[0].resize(F.n);
    std::vector<int> count(n_groups, 0);
    for (int64_t c = 0; c < F.n; ++c) {
      const int g = group_of_cell[F.iperm[c]];
      if (g < 0 || g >= n_groups) throw ArgError("group id out of range");
      grp[0][c] = g;
      count[g]++;
    }
    for (int g = 0; g < n_groups; ++g)
      if (count[g] == 0) throw ArgError("empty group");
    for (int l = 1; l < M.nlev; ++l) {
      const CoarseLevel& C = M.H.coarse[l - 1];
      grp[l].assign(C.n, -1);
      for (int64_t i = 0; i < (int64_t)grp[l - 1].size(); ++i) {
        const int64_t I = C.parent_of_fine[i];
        if (grp[l][I] >= 0 && grp[l][I] != grp[l - 1][i]) throw ArgError("a coarse cell spans two groups");
        grp[l][I] = grp[l - 1][i];
      }
    }
    M.gpool.clear();
    M.lgrp.assign(M.nlev, nullptr);
    for (int l = 0; l < M.nlev; ++l) {
      M.lgrp[l] = upload(M.gpool, grp[l]);
      M.lev[l].faces.grp = M.lgrp[l];
    }
    M.fine.grp = M.lgrp[0];
    // fine cells of each group in colour order
    std::vector<int> off(n_groups + 1, 0), idx(F.n);
    for (int g = 0; g < n_groups; ++g) off[g + 1] = off[g] + count[g];
    std::vector<int> pos(off.begin(), off.end() - 1);
    for (int64_t c = 0; c < F.n; ++c) idx[pos[grp[0][c]]++] = (int)c;
    M.goff = upload(M.gpool, off);
    M.gidx = upload(M.gpool, idx);
    M.qcell = dalloc<double>(M.gpool, (size_t)F.n * 2 * nv);
    M.hist_g = dalloc<double>(M.gpool, (size_t)M.max_hist * n_groups * 2 * nv);
    M.last_g = dalloc<double>(M.gpool, (size_t)n_groups * 2 * nv);
    M.active = upload(M.gpool, std::vector<int>(n_groups, 1));
    M.gcount = count;
    M.n_groups = n_groups;
    M.winf_h.assign(winf, winf + (size_t)n_groups * nv);
    DBuf* wb = new DBuf;
    M.gpool.emplace_back(wb);
    wb->alloc((size_t)n_groups * nv * sizeof(double));
    CK(cudaMemcpy(wb->p, winf, (size_t)n_groups * nv * sizeof(double), cudaMemcpyHostToDevice));
    M.winf = wb->as<double>();
    M.drop_graphs();
    CK(cudaDeviceSynchronize());
    return CGKS_OK;
  });
}

int cgks_vcycle_groups(cgks_t* h, int mesh_id, int n_cycles, int mode, double* norms_out, int* cycles_to_tol,
                       int* cycles_done) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (M.lgrp.empty()) throw StateError("cgks_set_groups has not been called for this mesh");
    if (n_cycles < 0 || (mode != CGKS_PLAIN_FP64 && mode != CGKS_MIXED)) throw ArgError("invalid arguments");
    const int G = M.n_groups, nv = M.nv;
    cudaGraphExec_t g = get_graph(h, M, mode);
    int start = 0;
    CK(cudaMemcpyAsync(&start, M.cycle, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<int> act(G, 1), conv(G, -1);
    std::vector<double> hist, first(G, -1.0);
    int done = 0, status = CGKS_OK;
    CK(cudaMemcpyAsync(M.active, act.data(), G * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    while (done < n_cycles) {
      const int chunk = std::min(h->cfg.check_every, n_cycles - done);
      for (int i = 0; i < chunk; ++i) CK(cudaGraphLaunch(g, h->stream));
      const int upto = std::min(start + done + chunk, M.max_hist);
      hist.resize((size_t)upto * G * 2 * nv);
      CK(cudaMemcpyAsync(hist.data(), M.hist_g, hist.size() * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      for (int k = start + done; k < upto; ++k)
        for (int q = 0; q < G; ++q) {
          const double r = hist[((size_t)k * G + q) * 2 * nv];
          if (first[q] < 0) first[q] = r;
          if (!act[q]) continue;
          if (!std::isfinite(r) || (first[q] > 0 && r > h->cfg.diverge_factor * first[q])) {
            // diverged: freeze this member and carry on with the others
            status = CGKS_ERR_DIVERGED;
            conv[q] = -2;
            act[q] = 0;
          } else if (conv[q] < 0 && first[q] > 0 && r <= h->cfg.tol * first[q]) {
            conv[q] = k - start + 1;
            act[q] = 0;  // converged: freeze this member
          }
        }
      done += chunk;
      CK(cudaMemcpyAsync(M.active, act.data(), G * sizeof(int), cudaMemcpyHostToDevice, h->stream));
      if (std::all_of(act.begin(), act.end(), [](int a) { return a == 0; })) break;
    }
    std::fill(act.begin(), act.end(), 1);
    CK(cudaMemcpyAsync(M.active, act.data(), G * sizeof(int), cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (norms_out)
      for (int i = 0; i < n_cycles; ++i)
        for (int j = 0; j < G * 2 * nv; ++j) {
          const size_t idx = (size_t)(start + i) * G * 2 * nv + j;
          norms_out[(size_t)i * G * 2 * nv + j] = (i < done && start + i < M.max_hist) ? hist[idx] : -1.0;
        }
    if (cycles_to_tol) std::memcpy(cycles_to_tol, conv.data(), G * sizeof(int));
    if (cycles_done) *cycles_done = done;
    if (status != CGKS_OK) {
      h->err = "batch members diverged (frozen, the others ran on):";
      for (int q = 0; q < G; ++q)
        if (conv[q] == -2) h->err += " " + std::to_string(q);
    }
    return status;
  });
}

int cgks_autotune(cgks_t* h, int mesh_id, int* blocks_out) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    const int cand[3] = {64, 128, 256};
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    auto timeit = [&](auto&& launch) {
      launch();
      CK(cudaEventRecord(e0, h->stream));
      for (int r = 0; r < 5; ++r) launch();
      CK(cudaEventRecord(e1, h->stream));
      CK(cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      return ms;
    };
    // populate R, D, face data at the current state (no state change)
    if (M.dim == 2) fine_residual<2>(h, M, false, true, false, false, M.gradnew, nullptr);
    else fine_residual<3>(h, M, false, true, false, false, M.gradnew, nullptr);
    LevelDev& L = M.lev[0];
    auto tune = [&](int cls, auto&& launch) {
      float best = 1e30f;
      int bb = M.blk[cls];
      for (int b : cand) {
        M.blk[cls] = b;
        const float t = timeit(launch);
        if (t < best) { best = t; bb = b; }
      }
      M.blk[cls] = bb;
    };
    const PhysParams p = phys(h->cfg, M.dim);
    if (M.dim == 2) {
      tune(B_RECON, [&] { launch_recon<2>(h, M); });
      tune(B_FLUX, [&] { launch_flux<2>(h, M); });
      tune(B_SWEEP, [&] {
        k_sweep<2, float, 0><<<blocks_for(L.color_off[1], M.blk[B_SWEEP]), M.blk[B_SWEEP], 0, h->stream>>>(
            L.topo, 0, L.color_off[1], L.W, L.R, nullptr, L.alpha, L.D, L.rface, h->cfg.gamma, L.dWs32, L.dW32);
      });
      if (M.nlev > 1) {
        LevelDev& C = M.lev[1];
        tune(B_FACE, [&] {
          k_face_kfvs<2><<<blocks_for(C.faces.nf, M.blk[B_FACE]), M.blk[B_FACE], 0, h->stream>>>(C.faces, C.W, M.winf, p, C.Fc, C.rface);
        });
        tune(B_CELL, [&] {
          k_coarse_cell<2, double><<<blocks_for(C.n, M.blk[B_CELL]), M.blk[B_CELL], 0, h->stream>>>(C.topo, C.W, C.Fc, C.rface, nullptr, nullptr, C.alpha, h->cfg.gamma, h->cfg.cfl_exp, h->cfg.cfl_imp, C.R, C.D, nullptr, nullptr, 0);
        });
      }
    } else {
      tune(B_RECON, [&] { launch_recon<3>(h, M); });
      tune(B_FLUX, [&] { launch_flux<3>(h, M); });
      tune(B_SWEEP, [&] {
        k_sweep<3, float, 0><<<blocks_for(L.color_off[1], M.blk[B_SWEEP]), M.blk[B_SWEEP], 0, h->stream>>>(
            L.topo, 0, L.color_off[1], L.W, L.R, nullptr, L.alpha, L.D, L.rface, h->cfg.gamma, L.dWs32, L.dW32);
      });
      if (M.nlev > 1) {
        LevelDev& C = M.lev[1];
        tune(B_FACE, [&] {
          k_face_kfvs<3><<<blocks_for(C.faces.nf, M.blk[B_FACE]), M.blk[B_FACE], 0, h->stream>>>(C.faces, C.W, M.winf, p, C.Fc, C.rface);
        });
        tune(B_CELL, [&] {
          k_coarse_cell<3, double><<<blocks_for(C.n, M.blk[B_CELL]), M.blk[B_CELL], 0, h->stream>>>(C.topo, C.W, C.Fc, C.rface, nullptr, nullptr, C.alpha, h->cfg.gamma, h->cfg.cfl_exp, h->cfg.cfl_imp, C.R, C.D, nullptr, nullptr, 0);
        });
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    CK(cudaGetLastError());
    M.drop_graphs();
    if (blocks_out)
      for (int i = 0; i < 7; ++i) blocks_out[i] = M.blk[i];
    return CGKS_OK;
  });
}

int cgks_kfvs_points(cgks_t* h, int dim, int64_t n, const double* Wl, const double* Wr, double* F) {
  return guarded(h, [&]() -> int {
    if ((dim != 2 && dim != 3) || n < 0 || n >= (1ll << 31) || !Wl || !Wr || !F) throw ArgError("invalid KFVS arguments");
    if (n == 0) return CGKS_OK;
    const PhysParams p = phys(h->cfg, dim);
    if (dim == 2) k_kfvs_points<2><<<blocks_for(n), kBlock, 0, h->stream>>>((int)n, p, Wl, Wr, F);
    else k_kfvs_points<3><<<blocks_for(n), kBlock, 0, h->stream>>>((int)n, p, Wl, Wr, F);
    CK(cudaGetLastError());
    return CGKS_OK;
  });
}

}  // extern "C"

// ===========================================================================
// Learned coarse-grid correction: network parameters, inference, gradients,
// training set and training loop.
// ===========================================================================
namespace cgks {
namespace {

using namespace cgks::mlp;

void mlp_ensure(cgks_t* h) {
  MlpState& S = h->mlp;
  if (S.ready) return;
  S.theta = dalloc<float>(S.pool, kParams);
  S.m = dalloc<float>(S.pool, kParams);
  S.v = dalloc<float>(S.pool, kParams);
  S.grad = dalloc<float>(S.pool, kParams);
  S.theta_bf = dalloc<__nv_bfloat16>(S.pool, kParams);
  S.tc_err = dalloc<int>(S.pool, 1);
  CK(cudaMemsetAsync(S.tc_err, 0, sizeof(int), h->stream));
  if (!S.tc_attr) {
    CK(cudaFuncSetAttribute(k_mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem));
    int occ = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_mlp_forward_tc, kTcThreads, kTcSmem));
    S.tc_blocks = std::max(1, occ) * h->sms;
    S.tc_attr = true;
  }
  S.ready = true;
}

void mlp_work(cgks_t* h, int64_t rows) {
  MlpState& S = h->mlp;
  if (rows <= S.work_rows) return;
  CK(cudaStreamSynchronize(h->stream));
  S.work.clear();
  S.work_rows = rows;
  auto& P = S.work;
  S.Z1 = dalloc<float>(P, rows * kH);
  S.Z2 = dalloc<float>(P, rows * kH);
  S.P = dalloc<float>(P, rows * kOut);
  S.dP = dalloc<float>(P, rows * kOut);
  S.A1 = dalloc<__nv_bfloat16>(P, rows * kH);
  S.A2 = dalloc<__nv_bfloat16>(P, rows * kH);
  S.dPb = dalloc<__nv_bfloat16>(P, rows * kOut);
  S.dZ2 = dalloc<__nv_bfloat16>(P, rows * kH);
  S.dZ1 = dalloc<__nv_bfloat16>(P, rows * kH);
  S.Xb = dalloc<__nv_bfloat16>(P, rows * kIn);
  S.Yb = dalloc<float>(P, rows * kOut);
  S.idx = dalloc<int>(P, rows);
  S.part = dalloc<float>(P, blocks_for(rows * kOut) + 1);
  S.loss = dalloc<float>(P, 1);
  S.split_elems = (size_t)64 * kH * kIn;
  S.split = dalloc<float>(P, S.split_elems);
}

void gemm(cudaStream_t st, const GemmArgs& g, int slices = 1) {
  dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, slices);
  k_gemm_bf16<<<grid, 128, 0, st>>>(g);
}

GemmArgs gargs(int M, int N, int K, const __nv_bfloat16* A, int lda, int ta, const __nv_bfloat16* B, int ldb,
               int tb, float* C, const float* bias, __nv_bfloat16* Abf, const float* Z, int epi) {
  GemmArgs g;
  g.M = M; g.N = N; g.K = K; g.A = A; g.lda = lda; g.ta = ta; g.B = B; g.ldb = ldb; g.tb = tb;
  g.C = C; g.bias = bias; g.Abf = Abf; g.Z = Z; g.epi = epi; g.k_per_slice = K;
  return g;
}

// forward pass on rows of X (bf16 [rows][68]) -> P (fp32 [rows][4]); keeps Z1, A1, Z2, A2
// for the backward pass when keep (the mma.sync chain always keeps them)
void mlp_forward(cgks_t* h, int64_t rows, const __nv_bfloat16* X, float* P, bool keep = true) {
  MlpState& S = h->mlp;
  const __nv_bfloat16* W = S.theta_bf;
  const int M = (int)rows;
  if (S.impl == 0) {
    const int ntiles = (int)((rows + kTcRows - 1) / kTcRows);
    const int nb = std::min(ntiles, S.tc_blocks);  // persistent: CTAs loop over the tiles
    k_mlp_forward_tc<<<nb, kTcThreads, kTcSmem, h->stream>>>(M, X, W, S.theta, keep ? S.Z1 : nullptr,
                                                            keep ? S.A1 : nullptr, keep ? S.Z2 : nullptr,
                                                            keep ? S.A2 : nullptr, P, S.tc_err);
    return;
  }
  gemm(h->stream, gargs(M, kH, kIn, X, kIn, 0, W + oW1, kIn, 1, S.Z1, S.theta + ob1, S.A1, nullptr, kEpiGeluBf16));
  gemm(h->stream, gargs(M, kH, kH, S.A1, kH, 0, W + oW2, kH, 1, S.Z2, S.theta + ob2, S.A2, nullptr, kEpiGeluBf16));
  gemm(h->stream, gargs(M, kOut, kH, S.A2, kH, 0, W + oW3, kH, 1, P, S.theta + ob3, nullptr, nullptr, kEpiStore));
}

// split-K weight gradient G[M][N] = op(A)^T-style product over K = rows
void grad_gemm(cgks_t* h, int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
               float* G) {
  MlpState& S = h->mlp;
  int slices = std::max(1, std::min(64, (K + 1023) / 1024));
  int kps = (K + slices - 1) / slices;
  kps = (kps + 15) / 16 * 16;
  slices = (K + kps - 1) / kps;
  GemmArgs g = gargs(M, N, K, A, lda, 1, B, ldb, 0, S.split, nullptr, nullptr, nullptr, kEpiPartial);
  g.k_per_slice = kps;
  gemm(h->stream, g, slices);
  k_reduce_slices<<<blocks_for((int64_t)M * N), kBlock, 0, h->stream>>>(S.split, slices, M * N, G);
}

// loss and gradient of the mean squared error at rows (X, Y) -> S.grad, S.loss
void mlp_backward(cgks_t* h, int64_t rows, const __nv_bfloat16* X, const float* Y) {
  MlpState& S = h->mlp;
  const int M = (int)rows;
  mlp_forward(h, rows, X, S.P);
  const int n = M * kOut;
  const int nb = (int)blocks_for(n);
  k_mse_grad<<<nb, kBlock, 0, h->stream>>>(S.P, Y, n, 1.0f / n, S.dP, S.dPb, S.part);
  k_sum_fixed<<<1, kBlock, 0, h->stream>>>(S.part, nb, 1.0f / n, S.loss);
  const __nv_bfloat16* W = S.theta_bf;
  float* g = S.grad;
  // layer 3
  grad_gemm(h, kOut, kH, M, S.dPb, kOut, S.A2, kH, g + oW3);
  k_colsum<float><<<kOut, kBlock, 0, h->stream>>>(S.dP, M, kOut, g + ob3);
  // dZ2 = (dP W3) * gelu'(Z2)
  gemm(h->stream, gargs(M, kH, kOut, S.dPb, kOut, 0, W + oW3, kH, 0, nullptr, nullptr, S.dZ2, S.Z2, kEpiGeluGrad));
  grad_gemm(h, kH, kH, M, S.dZ2, kH, S.A1, kH, g + oW2);
  k_colsum<__nv_bfloat16><<<kH, kBlock, 0, h->stream>>>(S.dZ2, M, kH, g + ob2);
  // dZ1 = (dZ2 W2) * gelu'(Z1)
  gemm(h->stream, gargs(M, kH, kH, S.dZ2, kH, 0, W + oW2, kH, 0, nullptr, nullptr, S.dZ1, S.Z1, kEpiGeluGrad));
  grad_gemm(h, kH, kIn, M, S.dZ1, kH, X, kIn, g + oW1);
  k_colsum<__nv_bfloat16><<<kH, kBlock, 0, h->stream>>>(S.dZ1, M, kH, g + ob1);
}

void ensure_learned(cgks_t* h, MeshDev& M) {
  if (M.dim != 2) throw ArgError("the learned correction is implemented for 2-D meshes");
  if (!h->mlp.ready) throw StateError("cgks_mlp_set_params has not been called");
  const int64_t n = M.lev[0].n;
  if (!M.X) {
    M.X = dalloc<__nv_bfloat16>(M.lpool, n * kIn);
    M.Pl = dalloc<float>(M.lpool, n * kOut);
    M.Yl = dalloc<float>(M.lpool, n * kOut);
    M.Wsave = dalloc<double>(M.lpool, n * M.nv);
    M.Sl = dalloc<float>(M.lpool, n);
    M.judge_part = dalloc<double>(M.lpool, 8 * blocks_for(n));
    M.judge_out = dalloc<double>(M.lpool, 8);
    if (M.nlev >= 3) {
      M.Rp1 = dalloc<double>(M.lpool, (size_t)M.lev[1].n * 4);
      M.Rp2 = dalloc<double>(M.lpool, (size_t)M.lev[2].n * 4);
    }
  }
  mlp_work(h, n);
}

static_assert(kFeat == kIn, "network input width");

void features(cgks_t* h, MeshDev& M) {
  LevelDev& L = M.lev[0];
  const bool coarse = M.nlev >= 3;
  if (coarse) {
    LevelDev& C1 = M.lev[1];
    LevelDev& C2 = M.lev[2];
    k_sum_children<<<blocks_for(C1.n), kBlock, 0, h->stream>>>(C1.n, C1.ch_off, C1.ch_idx, L.R, M.Rp1);
    k_sum_children<<<blocks_for(C2.n), kBlock, 0, h->stream>>>(C2.n, C2.ch_off, C2.ch_idx, M.Rp1, M.Rp2);
  }
  k_features2<<<blocks_for(L.n), kBlock, 0, h->stream>>>(
      M.fine, L.W, M.G, L.R, L.dti, L.alpha, M.winf, h->cfg.gamma, coarse ? L.parent : nullptr,
      coarse ? M.lev[1].parent : nullptr, M.Rp1, M.Rp2, coarse ? M.lev[1].vol : nullptr,
      coarse ? M.lev[2].vol : nullptr, M.lgrp.empty() ? M.last_norm : M.last_g, M.X,
      h->cfg.learned_scale ? M.Sl : nullptr);
}

template <typename T>
void enqueue_learned(cgks_t* h, MeshDev& M, bool judge) {
  LevelDev& L = M.lev[0];
  vcycle_pre<2, T>(h, M);
  features(h, M);
  mlp_forward(h, L.n, M.X, M.Pl, false);
  const int* grp = M.lgrp.empty() ? nullptr : M.lgrp[0];
  if (!judge) {
    k_apply_learned2<<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.n, M.Pl, L.alpha, h->cfg.df_gate, grp, M.winf,
                                                                 M.lgrp.empty() ? nullptr : M.active, h->cfg.gamma,
                                                                 h->cfg.learned_scale ? M.Sl : nullptr, L.W, M.cnt);
    return;
  }
  CK(cudaMemcpyAsync(M.Wsave, L.W, (size_t)L.n * M.nv * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  vcycle_coarse<2, T>(h, M);
  const int nb = (int)blocks_for(L.n);
  k_judge2<<<nb, kBlock, 0, h->stream>>>(L.n, M.Pl, L.W, M.Wsave, L.alpha, h->cfg.df_gate, grp, M.winf, h->cfg.gamma,
                                         h->cfg.learned_scale ? M.Sl : nullptr, M.judge_part);
  k_judge_final<<<1, 32, 0, h->stream>>>(M.judge_part, nb, M.judge_out);
}

void enqueue_kind(cgks_t* h, MeshDev& M, int kind, int prec) {
  if (kind == 0) {
    if (M.dim == 2) {
      if (prec == CGKS_MIXED) vcycle_body<2, float>(h, M);
      else vcycle_body<2, double>(h, M);
    } else {
      if (prec == CGKS_MIXED) vcycle_body<3, float>(h, M);
      else vcycle_body<3, double>(h, M);
    }
    return;
  }
  if (!M.X || h->mlp.work_rows < M.lev[0].n) throw StateError("learned buffers missing");
  if (prec == CGKS_MIXED) enqueue_learned<float>(h, M, kind == 2);
  else enqueue_learned<double>(h, M, kind == 2);
}

}  // namespace
}  // namespace cgks

extern "C" {

int cgks_mlp_features(cgks_t* h, int mesh_id, uint16_t* X_out) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (!X_out) throw ArgError("null output");
    ensure_learned(h, M);
    LevelDev& L = M.lev[0];
    // residual, time steps and DF at the current state (slopes unchanged);
    // with learned_scale 1 also its norms, which set the inputs' scale
    fine_residual<2>(h, M, false, false, h->cfg.learned_scale != 0, false, nullptr, nullptr);
    features(h, M);
    std::vector<uint16_t> tmp((size_t)L.n * kIn);
    CK(cudaMemcpyAsync(tmp.data(), M.X, tmp.size() * sizeof(uint16_t), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    const auto& iperm = M.H.fine.iperm;
    for (int64_t i = 0; i < L.n; ++i)
      std::memcpy(X_out + (size_t)iperm[i] * kIn, tmp.data() + (size_t)i * kIn, kIn * sizeof(uint16_t));
    return CGKS_OK;
  });
}

int cgks_mlp_collect(cgks_t* h, int mesh_id, int n_cycles, int mode) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    require_ready(M, true);
    if (n_cycles < 0 || (mode != CGKS_PLAIN_FP64 && mode != CGKS_MIXED)) throw ArgError("invalid arguments");
    if (M.nlev < 2) throw StateError("a coarse level is needed to produce corrections");
    ensure_learned(h, M);
    LevelDev& L = M.lev[0];
    const int* grp = M.lgrp.empty() ? nullptr : M.lgrp[0];
    for (int k = 0; k < n_cycles; ++k) {
      if (mode == CGKS_MIXED) vcycle_pre<2, float>(h, M);
      else vcycle_pre<2, double>(h, M);
      features(h, M);
      CK(cudaMemcpyAsync(M.Wsave, L.W, (size_t)L.n * M.nv * sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
      if (mode == CGKS_MIXED) vcycle_coarse<2, float>(h, M);
      else vcycle_coarse<2, double>(h, M);
      k_target2<<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.n, L.W, M.Wsave, grp, M.winf, h->cfg.gamma,
                                                           h->cfg.learned_scale ? M.Sl : nullptr, M.Yl);
      CK(cudaGetLastError());
      const int rc = cgks_mlp_dataset_append(h, L.n, (const uint16_t*)M.X, M.Yl);
      if (rc != CGKS_OK) return rc;
    }
    return CGKS_OK;
  });
}

int cgks_learned_stats(cgks_t* h, int mesh_id, double* out) {
  return guarded(h, [&]() -> int {
    MeshDev& M = get_mesh(h, mesh_id);
    if (!out) throw ArgError("null output");
    for (int i = 0; i < 10; ++i) out[i] = M.lstats[i];
    return CGKS_OK;
  });
}

}  // extern "C"

extern "C" {

int cgks_mlp_set_params(cgks_t* h, const float* theta) {
  return guarded(h, [&]() -> int {
    if (!theta) throw ArgError("null parameters");
    mlp_ensure(h);
    MlpState& S = h->mlp;
    CK(cudaMemcpyAsync(S.theta, theta, kParams * sizeof(float), cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemsetAsync(S.m, 0, kParams * sizeof(float), h->stream));
    CK(cudaMemsetAsync(S.v, 0, kParams * sizeof(float), h->stream));
    k_f32_to_bf16<<<blocks_for(kParams), kBlock, 0, h->stream>>>(kParams, S.theta, S.theta_bf);
    S.step = 0;
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_mlp_get_params(cgks_t* h, float* theta) {
  return guarded(h, [&]() -> int {
    if (!theta || !h->mlp.ready) throw StateError("no network parameters");
    CK(cudaMemcpyAsync(theta, h->mlp.theta, kParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    return CGKS_OK;
  });
}

int cgks_mlp_forward(cgks_t* h, int64_t n, const uint16_t* X, float* P) {
  return guarded(h, [&]() -> int {
    if (n <= 0 || n > (1ll << 30) || !X || !P) throw ArgError("invalid forward arguments");
    if (!h->mlp.ready) throw StateError("no network parameters");
    mlp_work(h, n);
    mlp_forward(h, n, (const __nv_bfloat16*)X, P, false);
    CK(cudaGetLastError());
    return CGKS_OK;
  });
}

int cgks_mlp_select(cgks_t* h, int impl) {
  return guarded(h, [&]() -> int {
    if (impl != 0 && impl != 1) throw ArgError("impl must be 0 (tcgen05) or 1 (mma.sync)");
    if (h->mlp.impl != impl) {
      h->mlp.impl = impl;
      for (auto& kv : h->meshes) kv.second->drop_graphs();  // learned graphs hold the old kernels
    }
    return CGKS_OK;
  });
}

int cgks_mlp_grad(cgks_t* h, int64_t n, const uint16_t* X, const float* Y, float* grad, float* loss) {
  return guarded(h, [&]() -> int {
    if (n <= 0 || n > (1ll << 30) || !X || !Y || !grad) throw ArgError("invalid gradient arguments");
    if (!h->mlp.ready) throw StateError("no network parameters");
    mlp_work(h, n);
    mlp_backward(h, n, (const __nv_bfloat16*)X, Y);
    CK(cudaMemcpyAsync(grad, h->mlp.grad, kParams * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
    if (loss) {
      CK(cudaMemcpyAsync(loss, h->mlp.loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaStreamSynchronize(h->stream));
    }
    CK(cudaGetLastError());
    return CGKS_OK;
  });
}

int cgks_mlp_dataset_append(cgks_t* h, int64_t n, const uint16_t* X, const float* Y) {
  return guarded(h, [&]() -> int {
    if (n <= 0 || !X || !Y) throw ArgError("invalid dataset arguments");
    MlpState& S = h->mlp;
    if (S.rows + n > S.cap) {
      const int64_t cap = std::max<int64_t>(S.rows + n, 2 * S.cap);
      std::vector<std::unique_ptr<DBuf>> nd;
      __nv_bfloat16* X2 = dalloc<__nv_bfloat16>(nd, cap * kIn);
      float* Y2 = dalloc<float>(nd, cap * kOut);
      if (S.rows) {
        CK(cudaMemcpyAsync(X2, S.X, S.rows * kIn * sizeof(__nv_bfloat16), cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaMemcpyAsync(Y2, S.Y, S.rows * kOut * sizeof(float), cudaMemcpyDeviceToDevice, h->stream));
      }
      CK(cudaStreamSynchronize(h->stream));
      S.data = std::move(nd);
      S.X = X2;
      S.Y = Y2;
      S.cap = cap;
    }
    CK(cudaMemcpyAsync(S.X + S.rows * kIn, X, n * kIn * sizeof(__nv_bfloat16), cudaMemcpyDefault, h->stream));
    CK(cudaMemcpyAsync(S.Y + S.rows * kOut, Y, n * kOut * sizeof(float), cudaMemcpyDefault, h->stream));
    // rows with a non-finite input or target (a diverging mesh) take no part in training
    k_mark_nonfinite_rows<<<blocks_for(n), kBlock, 0, h->stream>>>(n, S.X + S.rows * kIn, S.Y + S.rows * kOut);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
    S.rows += n;
    return CGKS_OK;
  });
}

int cgks_mlp_dataset_size(cgks_t* h, int64_t* n) {
  return guarded(h, [&]() -> int {
    if (!n) throw ArgError("null output");
    *n = h->mlp.rows;
    return CGKS_OK;
  });
}

int cgks_mlp_dataset_clear(cgks_t* h) {
  return guarded(h, [&]() -> int {
    CK(cudaStreamSynchronize(h->stream));
    h->mlp.data.clear();
    h->mlp.X = nullptr;
    h->mlp.Y = nullptr;
    h->mlp.rows = h->mlp.cap = 0;
    return CGKS_OK;
  });
}

int cgks_mlp_train(cgks_t* h, int n_steps, int batch, double lr, uint64_t seed, float* losses) {
  return guarded(h, [&]() -> int {
    MlpState& S = h->mlp;
    if (n_steps < 0 || batch < 1 || !(lr > 0)) throw ArgError("invalid training arguments");
    if (!S.ready) throw StateError("no network parameters");
    if (S.rows < 1) throw StateError("empty training set");
    const int64_t b = std::min<int64_t>(batch, S.rows);
    mlp_work(h, b);
    std::vector<int> idx(b);
    uint64_t st = seed;
    auto next = [&]() {  // splitmix64
      st += 0x9E3779B97F4A7C15ull;
      uint64_t z = st;
      z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
      z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
      return z ^ (z >> 31);
    };
    std::vector<float> lh(n_steps);
    for (int s = 0; s < n_steps; ++s) {
      for (int64_t i = 0; i < b; ++i) idx[i] = (int)(next() % (uint64_t)S.rows);
      CK(cudaMemcpyAsync(S.idx, idx.data(), b * sizeof(int), cudaMemcpyHostToDevice, h->stream));
      k_gather_batch<<<blocks_for(b * kIn), kBlock, 0, h->stream>>>((int)b, S.idx, S.X, S.Y, S.Xb, S.Yb);
      mlp_backward(h, b, S.Xb, S.Yb);
      S.step++;
      const float b1 = 0.9f, b2 = 0.999f;
      k_adam<<<blocks_for(kParams), kBlock, 0, h->stream>>>(kParams, S.grad, S.theta, S.m, S.v, S.theta_bf,
                                                             (float)lr, b1, b2, 1e-8f,
                                                             1.f - std::pow(b1, (float)S.step),
                                                             1.f - std::pow(b2, (float)S.step));
      if (losses) CK(cudaMemcpyAsync(&lh[s], S.loss, sizeof(float), cudaMemcpyDeviceToHost, h->stream));
      // the host index buffer is reused next step: wait for this step's copy
      CK(cudaStreamSynchronize(h->stream));
    }
    if (losses) std::memcpy(losses, lh.data(), n_steps * sizeof(float));
    CK(cudaGetLastError());
    check_tc_error(h);
    return CGKS_OK;
  });
}

}  // extern "C"

// ===========================================================================
// Coarse KFVS residual without any allocation.
//
// Some callers cannot let a library call allocate device memory: for example
// an application that pre-plans every byte of the GPU before its time loop, or
// a caller on a latency-critical path where cudaMalloc / cudaFree would add an
// implicit device-wide synchronisation.  This variant of the coarse residual
// (cgks_residual with level >= 1) therefore keeps its only scratch buffer, the
// per-face flux, in a fixed device array that lives in this library from load
// to process exit, and reads and writes the caller's buffers directly.
// ===========================================================================
namespace cgks {
namespace noalloc {

// Capacity of the face-flux scratch: 131,072 faces x 5 conservative variables
// of FP64 (5 MiB).  Every GPU that loads the library holds this array.
constexpr int kNoAllocMaxFaces = 131072;
static __device__ __align__(256) double g_noalloc_face_flux[kNoAllocMaxFaces * 5];

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_noalloc_face(FaceSet Fs, const int* __restrict__ iperm,
                                                         const double* __restrict__ W_orig,
                                                         const double* __restrict__ winf, PhysParams P,
                                                         double* __restrict__ Fout) {
  constexpr int NV = DIM + 2;
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= Fs.nf) return;
  const int L = Fs.fL[f], R = Fs.fR[f];
  double n[DIM], WL[NV], WR[NV];
#pragma unroll
  for (int d = 0; d < DIM; ++d) n[d] = Fs.fn[(size_t)f * DIM + d];
#pragma unroll
  for (int v = 0; v < NV; ++v) WL[v] = W_orig[(size_t)iperm[L] * NV + v];
  if (R >= 0) {
#pragma unroll
    for (int v = 0; v < NV; ++v) WR[v] = W_orig[(size_t)iperm[R] * NV + v];
  } else {
    ghost_state<DIM>(Fs.ftag[f], winf + NV * (Fs.grp ? Fs.grp[L] : 0), n, WL, WR, P.gamma);
  }
  const Frame<DIM> fr = make_frame<DIM>(n);
  double wl[NV], wr[NV], Fl[NV], Fg[NV];
  to_local<DIM>(fr, WL, wl);
  to_local<DIM>(fr, WR, wr);
  kfvs_flux<DIM>(P, wl, wr, Fl);
  to_global<DIM>(fr, Fl, Fg);
  const double S = Fs.fS[f];
#pragma unroll
  for (int v = 0; v < NV; ++v) Fout[(size_t)f * NV + v] = S * Fg[v];
}

template <int DIM>
__global__ void __launch_bounds__(kBlock) k_noalloc_cell(Topo Tp, const int* __restrict__ iperm,
                                                         const double* __restrict__ Fface,
                                                         double* __restrict__ R_orig) {
  constexpr int NV = DIM + 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Tp.n) return;
  double r[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) r[v] = 0.0;
  for (int e = Tp.off[c]; e < Tp.off[c + 1]; ++e) {
    const int f = Tp.face[e];
    const double sd = Tp.side[e];
#pragma unroll
    for (int v = 0; v < NV; ++v) r[v] += sd * Fface[(size_t)f * NV + v];
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) R_orig[(size_t)iperm[c] * NV + v] = r[v];
}

int noalloc_fail(cgks_t* h, int code, const char* msg) {
  h->err.assign(msg);  // within the capacity reserved at cgks_create
  return code;
}

// Error message naming the CUDA error, composed in a fixed buffer so that
// reporting a failure allocates nothing either.
int noalloc_cuda_fail(cgks_t* h, const char* what, cudaError_t e) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "cgks_residual_coarse_noalloc: %s: %s", what, cudaGetErrorString(e));
  return noalloc_fail(h, CGKS_ERR_CUDA, buf);
}

}  // namespace noalloc
}  // namespace cgks

using namespace cgks::noalloc;

extern "C" int cgks_residual_coarse_noalloc(cgks_t* h, int mesh_id, int level, const double* W_dev,
                                            double* R_dev) {
  if (!h) return CGKS_ERR_ARG;
  auto it = h->meshes.find(mesh_id);
  if (it == h->meshes.end()) return noalloc_fail(h, CGKS_ERR_ARG, "unknown mesh id");
  MeshDev& M = *it->second;
  if (!M.has_hierarchy || M.winf_h.empty())
    return noalloc_fail(h, CGKS_ERR_STATE, "mesh hierarchy or free stream not set");
  if (level < 1 || level >= M.nlev || !W_dev || !R_dev)
    return noalloc_fail(h, CGKS_ERR_ARG, "level must be a coarse level (>= 1) and buffers non-null");
  LevelDev& L = M.lev[level];
  if (L.faces.nf > kNoAllocMaxFaces)
    return noalloc_fail(h, CGKS_ERR_ARG,
                        "cgks_residual_coarse_noalloc: the level has more than 131072 faces, the capacity "
                        "of the fixed face-flux buffer; use cgks_residual instead");
  // All work runs on the context's device: make it current for this call and
  // put the caller's device back on every return path.
  int prev_dev = h->device;
  if (cudaGetDevice(&prev_dev) != cudaSuccess) prev_dev = h->device;
  if (prev_dev != h->device) {
    const cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return noalloc_cuda_fail(h, "cudaSetDevice to the context's device failed", e);
  }
  struct RestoreDevice {
    int prev, cur;
    ~RestoreDevice() {
      if (prev != cur) cudaSetDevice(prev);
    }
  } restore{prev_dev, h->device};
  if (!h->noalloc_scratch) {
    // First call on this context: the array's device address on the context's
    // device.  A context never outlives a device reset (its own buffers would
    // be gone too), so the address is looked up again by any new context.
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_face_flux);
    if (e != cudaSuccess) return noalloc_cuda_fail(h, "cudaGetSymbolAddress failed", e);
    h->noalloc_scratch = (double*)p;
  }
  double* scratch = h->noalloc_scratch;
  // every face entry the cell kernel reads is written by the face kernel first,
  // so the buffer needs no clearing between calls
  const PhysParams p = phys(h->cfg, M.dim);
  // a non-sticky error left by earlier, unrelated work on this thread is not
  // this call's failure: clear it so that the checks below see only these launches
  (void)cudaGetLastError();
  cudaError_t e;
  if (M.dim == 2)
    k_noalloc_face<2><<<blocks_for(L.faces.nf), kBlock, 0, h->stream>>>(L.faces, L.iperm, W_dev, M.winf, p, scratch);
  else
    k_noalloc_face<3><<<blocks_for(L.faces.nf), kBlock, 0, h->stream>>>(L.faces, L.iperm, W_dev, M.winf, p, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_cuda_fail(h, "face-flux kernel launch failed", e);
  if (M.dim == 2)
    k_noalloc_cell<2><<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.topo, L.iperm, scratch, R_dev);
  else
    k_noalloc_cell<3><<<blocks_for(L.n), kBlock, 0, h->stream>>>(L.topo, L.iperm, scratch, R_dev);
  if ((e = cudaGetLastError()) != cudaSuccess) return noalloc_cuda_fail(h, "cell-sum kernel launch failed", e);
  return CGKS_OK;
}
