// Host-side mesh preprocessing (see host_mesh.hpp).
#include "host_mesh.hpp"

#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <deque>
#include <stdexcept>
#include <unordered_map>

namespace cgks {
namespace {

struct FaceKey {
  std::array<int32_t, 3> v;
  bool operator==(const FaceKey& o) const { return v == o.v; }
};
struct FaceKeyHash {
  size_t operator()(const FaceKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 3; ++i) { h ^= (uint64_t)(uint32_t)k.v[i]; h *= 1099511628211ull; }
    return (size_t)h;
  }
};

FaceKey make_key(const int32_t* ids, int cnt) {
  FaceKey k{{-1, -1, -1}};
  for (int i = 0; i < cnt; ++i) k.v[i] = ids[i];
  std::sort(k.v.begin(), k.v.begin() + cnt);
  return k;
}

// index of X_p X_q (p <= q) among the quadratic monomials: xx, xy, yy or
// xx, xy, xz, yy, yz, zz
int qidx(int dim, int p, int q) {
  if (p > q) std::swap(p, q);
  if (dim == 2) return p == 0 ? q : 2;
  static const int t[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
  return t[p][q];
}

// Cholesky factorisation in place (lower); returns false if not positive definite
bool cholesky(std::vector<double>& A, int n, double rel_tol) {
  double dmax = 0.0;
  for (int i = 0; i < n; ++i) dmax = std::max(dmax, std::fabs(A[i * n + i]));
  for (int j = 0; j < n; ++j) {
    double d = A[j * n + j];
    for (int k = 0; k < j; ++k) d -= A[j * n + k] * A[j * n + k];
    if (!(d > rel_tol * dmax)) return false;
    d = std::sqrt(d);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[i * n + j];
      for (int k = 0; k < j; ++k) s -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = s / d;
    }
  }
  return true;
}
// X <- A^-1 X for a Cholesky factor L (A = L L^T), X has m columns
void chol_solve(const std::vector<double>& L, int n, std::vector<double>& X, int m) {
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < n; ++i) {
      double s = X[i * m + c];
      for (int k = 0; k < i; ++k) s -= L[i * n + k] * X[k * m + c];
      X[i * m + c] = s / L[i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = X[i * m + c];
      for (int k = i + 1; k < n; ++k) s -= L[k * n + i] * X[k * m + c];
      X[i * m + c] = s / L[i * n + i];
    }
  }
}

}  // namespace

int greedy_colouring(int64_t n, const std::vector<int64_t>& off, const std::vector<int64_t>& nbr,
                     std::vector<int32_t>& colour) {
  colour.assign(n, 0);
  std::deque<int64_t> queue;
  int nc = 0;
  int64_t painted = 0, scan = 0;
  auto paint = [&](int64_t w) {
    std::vector<char> used(8, 0);
    for (int64_t e = off[w]; e < off[w + 1]; ++e) {
      int64_t j = nbr[e];
      if (j < 0 || colour[j] == 0) continue;
      if ((size_t)colour[j] >= used.size()) used.resize(colour[j] + 1, 0);
      used[colour[j]] = 1;
    }
    int k = 1;
    while ((size_t)k < used.size() && used[k]) ++k;
    colour[w] = k;
    nc = std::max(nc, k);
    queue.push_back(w);
    ++painted;
  };
  while (painted < n) {
    while (scan < n && colour[scan] != 0) ++scan;
    paint(scan);  // start (or restart) at the lowest unpainted cell
    while (!queue.empty()) {
      int64_t v = queue.front();
      queue.pop_front();
      for (int64_t e = off[v]; e < off[v + 1]; ++e) {
        int64_t w = nbr[e];
        if (w >= 0 && colour[w] == 0) paint(w);
      }
    }
  }
  return nc;
}

namespace {

// stable colour-major renumbering
void renumber(const std::vector<int32_t>& colour, int nc, std::vector<int64_t>& perm,
              std::vector<int64_t>& iperm, std::vector<int64_t>& coff) {
  int64_t n = (int64_t)colour.size();
  coff.assign(nc + 1, 0);
  for (int64_t i = 0; i < n; ++i) coff[colour[i]]++;
  for (int c = 1; c <= nc; ++c) coff[c] += coff[c - 1];
  std::vector<int64_t> pos(coff.begin(), coff.end() - 1);
  perm.resize(n);
  iperm.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    int64_t p = pos[colour[i] - 1]++;
    perm[i] = p;
    iperm[p] = i;
  }
}

}  // namespace

namespace {

// A fine level before colouring, in the original cell numbering: cell
// geometry, each cell's faces in its stored order (padded to nfc entries),
// and per-face geometry with its Gauss points (padded to ngp points).
struct FineRaw {
  int dim = 0, nfc = 0, ngp = 0;
  int64_t n = 0, nf = 0, nf_int = 0;
  std::vector<double> vol, cen, m2;
  std::vector<int8_t> cnf;       // [n] faces of each cell
  std::vector<int64_t> ocface;   // [n][nfc] (-1 in the padding)
  std::vector<int8_t> ocside;    // [n][nfc]
  std::vector<int64_t> fL, fR;
  std::vector<int32_t> tag;
  std::vector<double> fnrm, fS;  // [nf][dim], [nf]
  std::vector<int8_t> fngp;      // [nf] Gauss points of each face
  std::vector<double> gp, gw;    // [nf][ngp][dim] points, [nf][ngp] weights (sum 1)
  std::vector<double> shift;     // [nf][dim] periodic shift (x seen from L minus from R)
  std::vector<double> fpt;       // [nf][dim] a point of the face plane (ghost mirror plane)
};

// Mixed meshes: faces with more Gauss points first, within the interior faces
// and within the boundary faces (a stable reorder), so that the 32 faces a warp
// of the flux kernel takes have one Gauss-point count except at the seams.
// Only the storage order changes: each cell still sums its faces in its own
// face order.
void group_faces_by_points(FineRaw& R) {
  const int64_t nf = R.nf, nf_int = R.nf_int;
  const int dim = R.dim, ngp = R.ngp;
  std::vector<int64_t> order(nf);
  for (int64_t f = 0; f < nf; ++f) order[f] = f;
  auto by_points = [&](int64_t a, int64_t b) { return R.fngp[a] > R.fngp[b]; };
  std::stable_sort(order.begin(), order.begin() + nf_int, by_points);
  std::stable_sort(order.begin() + nf_int, order.end(), by_points);
  std::vector<int64_t> newid(nf);
  for (int64_t f = 0; f < nf; ++f) newid[order[f]] = f;
  auto permute = [&](auto& v, int64_t w) {
    if (v.empty()) return;
    auto o = v;
    for (int64_t f = 0; f < nf; ++f)
      for (int64_t k = 0; k < w; ++k) v[f * w + k] = o[order[f] * w + k];
  };
  permute(R.fL, 1);
  permute(R.fR, 1);
  permute(R.tag, 1);
  permute(R.fnrm, dim);
  permute(R.fS, 1);
  permute(R.fngp, 1);
  permute(R.gp, (int64_t)ngp * dim);
  permute(R.gw, ngp);
  permute(R.shift, dim);
  permute(R.fpt, dim);
  for (auto& f : R.ocface)
    if (f >= 0) f = newid[f];
}

// Colouring, colour-major renumbering, faces and cells in the new numbering,
// and the per-cell reconstruction operator (Sec 3.1), shared by the simplex
// and the mixed-element meshes.
void finish_fine_level(FineRaw& R, bool mixed, FineLevel& F) {
  if (mixed) group_faces_by_points(R);
  const int dim = R.dim, nfc = R.nfc, ngp = R.ngp;
  const int64_t n = R.n, nf = R.nf, nf_int = R.nf_int;
  const std::vector<double>& vol = R.vol;
  const std::vector<double>& cen = R.cen;
  const std::vector<double>& m2 = R.m2;
  const std::vector<int64_t>& ocface = R.ocface;
  const std::vector<int8_t>& ocside = R.ocside;
  const std::vector<int64_t>& fL = R.fL;
  const std::vector<int64_t>& fR = R.fR;
  const std::vector<double>& fnrm = R.fnrm;
  const std::vector<double>& fS = R.fS;
  const std::vector<double>& gp = R.gp;
  const std::vector<double>& shift = R.shift;
  F.dim = dim; F.nv = dim + 2; F.ngp = ngp; F.nfc = nfc; F.nk = dim == 2 ? 5 : 9; F.n = n;
  F.mixed = mixed;
  // ---- colouring and renumbering ----------------------------------------
  {
    std::vector<int64_t> off(n + 1), nbr(n * nfc);
    for (int64_t c = 0; c <= n; ++c) off[c] = c * nfc;
    for (int64_t c = 0; c < n; ++c)
      for (int k = 0; k < nfc; ++k) {
        if (k >= R.cnf[c]) { nbr[c * nfc + k] = -1; continue; }
        int64_t f = ocface[c * nfc + k];
        nbr[c * nfc + k] = ocside[c * nfc + k] > 0 ? fR[f] : fL[f];
      }
    F.n_colors = greedy_colouring(n, off, nbr, F.color_orig);
    renumber(F.color_orig, F.n_colors, F.perm, F.iperm, F.color_off);
  }
  const auto& perm = F.perm;
  const auto& iperm = F.iperm;
  // ---- store faces with new cell ids -----------------------------------
  F.nf = nf; F.nf_int = nf_int;
  F.fL.resize(nf); F.fR.resize(nf); F.ftag = R.tag;
  F.fn = fnrm; F.fS = fS;
  F.XL.assign(nf * ngp * dim, 0.0); F.XR.assign(nf * ngp * dim, 0.0);
  if (mixed) { F.fngp = R.fngp; F.gw = R.gw; }
  for (int64_t f = 0; f < nf; ++f) {
    F.fL[f] = perm[fL[f]];
    F.fR[f] = fR[f] >= 0 ? perm[fR[f]] : -1;
    for (int g = 0; g < R.fngp[f]; ++g)
      for (int d = 0; d < dim; ++d) {
        double x = gp[(f * ngp + g) * dim + d];
        F.XL[(f * ngp + g) * dim + d] = x - cen[fL[f] * dim + d];
        if (fR[f] >= 0) F.XR[(f * ngp + g) * dim + d] = x - shift[f * dim + d] - cen[fR[f] * dim + d];
      }
  }
  // ---- cells in new order ------------------------------------------------
  F.vol.resize(n); F.cen.resize(n * dim); F.m2.resize(n * dim * dim);
  F.cface.assign(n * nfc, 0); F.cside.assign(n * nfc, 0); F.cnbr.assign(n * nfc, -1);
  if (mixed) F.cnf.resize(n);
  for (int64_t c = 0; c < n; ++c) {
    int64_t o = iperm[c];
    F.vol[c] = vol[o];
    for (int d = 0; d < dim; ++d) F.cen[c * dim + d] = cen[o * dim + d];
    for (int i = 0; i < dim * dim; ++i) F.m2[c * dim * dim + i] = m2[o * dim * dim + i];
    if (mixed) F.cnf[c] = R.cnf[o];
    for (int k = 0; k < R.cnf[o]; ++k) {
      int64_t f = ocface[o * nfc + k];
      F.cface[c * nfc + k] = f;
      F.cside[c * nfc + k] = ocside[o * nfc + k];
      int64_t j = ocside[o * nfc + k] > 0 ? fR[f] : fL[f];
      F.cnbr[c * nfc + k] = j >= 0 ? perm[j] : -1;
    }
  }
  // ---- reconstruction operator (constrained least squares, Sec 3.1) ------
  // Columns: nfc equality columns (the first ne used), then nfc * dim slope
  // columns (the first ne * dim used); ne = faces of the cell.
  const int nk = F.nk, ncol = nfc + nfc * dim;
  F.nop = nk * ncol;
  F.op.assign(n * F.nop, 0.0);
  F.op_ok.assign(n, 1);
  F.avg0.assign(n * nk, 0.0);
  F.gg.assign(n * nfc * dim, 0.0);
  std::vector<int> kp(nk), kq(nk);
  for (int k = 0; k < dim; ++k) { kp[k] = k; kq[k] = -1; }
  for (int p = 0; p < dim; ++p) for (int q = p; q < dim; ++q) { int k = dim + qidx(dim, p, q); kp[k] = p; kq[k] = q; }
  for (int64_t c = 0; c < n; ++c) {
    int64_t o = iperm[c];
    const int ne = R.cnf[o], nl = ne * dim;
    std::vector<double> C(ne * nk), B(nl * nk), H(nk * nk), Hl(nk * nk), Sm(ne * ne);
    const double* x0 = &cen[o * dim];
    const double* M0 = &m2[o * dim * dim];
    const double V0 = vol[o];
    const double h = std::pow(V0, 1.0 / dim);
    double a0[9];
    for (int k = 0; k < nk; ++k) a0[k] = kq[k] < 0 ? 0.0 : M0[kp[k] * dim + kq[k]];
    for (int k = 0; k < nk; ++k) F.avg0[c * nk + k] = a0[k];
    for (int m = 0; m < ne; ++m) {
      int64_t f = ocface[o * nfc + m];
      int side = ocside[o * nfc + m];
      double nn[3];
      for (int d = 0; d < dim; ++d) nn[d] = side * fnrm[f * dim + d];
      for (int d = 0; d < dim; ++d) F.gg[(c * nfc + m) * dim + d] = fS[f] * nn[d] / (2.0 * V0);
      // neighbour centroid and moments in cell o's frame
      double cm[3], Mm[9];
      int64_t j = side > 0 ? fR[f] : fL[f];
      if (j >= 0) {
        for (int d = 0; d < dim; ++d) cm[d] = cen[j * dim + d] + side * shift[f * dim + d];
        for (int i = 0; i < dim * dim; ++i) Mm[i] = m2[j * dim * dim + i];
      } else {
        // mirror image of cell o across the boundary face plane
        const double* xf = &R.fpt[f * dim];
        double hh = 0.0;
        for (int d = 0; d < dim; ++d) hh += (xf[d] - x0[d]) * nn[d];
        for (int d = 0; d < dim; ++d) cm[d] = x0[d] + 2.0 * hh * nn[d];
        for (int p = 0; p < dim; ++p)
          for (int q = 0; q < dim; ++q) {
            // (I - 2nn^T) M0 (I - 2nn^T)
            double s = 0.0;
            for (int r = 0; r < dim; ++r)
              for (int t = 0; t < dim; ++t)
                s += ((p == r) - 2.0 * nn[p] * nn[r]) * M0[r * dim + t] * ((t == q) - 2.0 * nn[t] * nn[q]);
            Mm[p * dim + q] = s;
          }
      }
      double dx[3];
      for (int d = 0; d < dim; ++d) dx[d] = cm[d] - x0[d];
      for (int k = 0; k < nk; ++k) {
        int p = kp[k], q = kq[k];
        double sc = q < 0 ? h : h * h;
        double am = q < 0 ? dx[p] : Mm[p * dim + q] + dx[p] * dx[q];
        C[m * nk + k] = (am - a0[k]) / sc;
        for (int d = 0; d < dim; ++d) {
          double da = q < 0 ? (d == p ? 1.0 : 0.0) : (d == p ? dx[q] : 0.0) + (d == q ? dx[p] : 0.0);
          B[(m * dim + d) * nk + k] = da / sc;
        }
      }
    }
    // a' = H^-1 B^T d + H^-1 C^T S^-1 (e - C H^-1 B^T d),  H = B^T B, S = C H^-1 C^T
    for (int i = 0; i < nk; ++i)
      for (int j = 0; j < nk; ++j) {
        double s = 0.0;
        for (int r = 0; r < nl; ++r) s += B[r * nk + i] * B[r * nk + j];
        H[i * nk + j] = s;
      }
    Hl = H;
    bool ok = cholesky(Hl, nk, 1e-13);
    std::vector<double> HiCt, HiBt, Sl;
    if (ok) {
      HiCt.assign(nk * ne, 0.0);
      for (int i = 0; i < nk; ++i) for (int m = 0; m < ne; ++m) HiCt[i * ne + m] = C[m * nk + i];
      chol_solve(Hl, nk, HiCt, ne);
      HiBt.assign(nk * nl, 0.0);
      for (int i = 0; i < nk; ++i) for (int r = 0; r < nl; ++r) HiBt[i * nl + r] = B[r * nk + i];
      chol_solve(Hl, nk, HiBt, nl);
      for (int a = 0; a < ne; ++a)
        for (int b = 0; b < ne; ++b) {
          double s = 0.0;
          for (int i = 0; i < nk; ++i) s += C[a * nk + i] * HiCt[i * ne + b];
          Sm[a * ne + b] = s;
        }
      Sl = Sm;
      ok = cholesky(Sl, ne, 1e-13);
    }
    if (!ok) { F.op_ok[c] = 0; continue; }
    // OpE = HiCt S^-1 ; OpD = HiBt - OpE (C HiBt)
    std::vector<double> Sinv(ne * ne, 0.0);
    for (int i = 0; i < ne; ++i) Sinv[i * ne + i] = 1.0;
    chol_solve(Sl, ne, Sinv, ne);
    std::vector<double> OpE(nk * ne, 0.0), CHB(ne * nl, 0.0);
    for (int i = 0; i < nk; ++i)
      for (int m = 0; m < ne; ++m) {
        double s = 0.0;
        for (int t = 0; t < ne; ++t) s += HiCt[i * ne + t] * Sinv[t * ne + m];
        OpE[i * ne + m] = s;
      }
    for (int m = 0; m < ne; ++m)
      for (int r = 0; r < nl; ++r) {
        double s = 0.0;
        for (int i = 0; i < nk; ++i) s += C[m * nk + i] * HiBt[i * nl + r];
        CHB[m * nl + r] = s;
      }
    double* op = &F.op[c * F.nop];
    for (int i = 0; i < nk; ++i) {
      double sc = kq[i] < 0 ? h : h * h;
      for (int m = 0; m < ne; ++m) op[i * ncol + m] = OpE[i * ne + m] / sc;
      for (int r = 0; r < nl; ++r) {
        double s = HiBt[i * nl + r];
        for (int m = 0; m < ne; ++m) s -= OpE[i * ne + m] * CHB[m * nl + r];
        op[i * ncol + nfc + r] = s / sc;
      }
    }
  }
}

}  // namespace

void build_fine_level(int dim, int64_t n, const int32_t* cn, const double* cx, int64_t nb,
                      const int32_t* bfn, const int32_t* bft, FineLevel& F) {
  if (dim != 2 && dim != 3) throw std::runtime_error("dim must be 2 or 3");
  if (n <= 0) throw std::runtime_error("mesh has no cells");
  const int nvert = dim + 1, nfc = dim + 1;
  F.dim = dim; F.nv = dim + 2; F.ngp = dim == 2 ? 2 : 3; F.nfc = nfc; F.nk = dim == 2 ? 5 : 9; F.n = n;
  // ---- geometry in original order -------------------------------------
  std::vector<double> vol(n), cen(n * dim), m2(n * dim * dim);
  for (int64_t c = 0; c < n; ++c) {
    const double* x = cx + c * nvert * dim;
    double det;
    if (dim == 2) {
      det = (x[2] - x[0]) * (x[5] - x[1]) - (x[3] - x[1]) * (x[4] - x[0]);
      vol[c] = 0.5 * std::fabs(det);
    } else {
      double a[3], b[3], d[3];
      for (int k = 0; k < 3; ++k) { a[k] = x[3 + k] - x[k]; b[k] = x[6 + k] - x[k]; d[k] = x[9 + k] - x[k]; }
      det = a[0] * (b[1] * d[2] - b[2] * d[1]) + a[1] * (b[2] * d[0] - b[0] * d[2]) + a[2] * (b[0] * d[1] - b[1] * d[0]);
      vol[c] = std::fabs(det) / 6.0;
    }
    if (!(vol[c] > 0.0)) throw std::runtime_error("degenerate cell " + std::to_string(c));
    for (int k = 0; k < dim; ++k) {
      double s = 0.0;
      for (int v = 0; v < nvert; ++v) s += x[v * dim + k];
      cen[c * dim + k] = s / nvert;
    }
    // central second moments by a degree-2 exact rule: edge midpoints (triangle),
    // symmetric 4-point rule (tetrahedron)
    double M[9] = {0};
    if (dim == 2) {
      for (int e = 0; e < 3; ++e) {
        double p[2];
        for (int k = 0; k < 2; ++k) p[k] = 0.5 * (x[e * 2 + k] + x[((e + 1) % 3) * 2 + k]) - cen[c * 2 + k];
        for (int i = 0; i < 2; ++i) for (int j = 0; j < 2; ++j) M[i * 2 + j] += p[i] * p[j] / 3.0;
      }
    } else {
      const double qa = 0.5854101966249685, qb = 0.1381966011250105;
      for (int q = 0; q < 4; ++q) {
        double p[3];
        for (int k = 0; k < 3; ++k) {
          double s = 0.0;
          for (int v = 0; v < 4; ++v) s += (v == q ? qa : qb) * x[v * 3 + k];
          p[k] = s - cen[c * 3 + k];
        }
        for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) M[i * 3 + j] += 0.25 * p[i] * p[j];
      }
    }
    for (int i = 0; i < dim * dim; ++i) m2[c * dim * dim + i] = M[i];
  }
  // ---- faces ----------------------------------------------------------
  std::unordered_map<FaceKey, int64_t, FaceKeyHash> bmap;
  bmap.reserve(nb * 2 + 1);
  for (int64_t b = 0; b < nb; ++b) {
    auto k = make_key(bfn + b * dim, dim);
    if (!bmap.emplace(k, b).second) throw std::runtime_error("duplicate boundary face");
  }
  std::unordered_map<FaceKey, int64_t, FaceKeyHash> open;  // key -> cell*nfc + k
  open.reserve(n * nfc);
  std::vector<int64_t> ocface(n * nfc, -1);
  std::vector<int8_t> ocside(n * nfc, 0);
  std::vector<int64_t> fL, fR;
  std::vector<int32_t> fk_l, fk_r;
  for (int64_t c = 0; c < n; ++c) {
    for (int k = 0; k < nfc; ++k) {
      int32_t ids[3];
      int m = 0;
      for (int v = 0; v < nvert; ++v) if (v != k) ids[m++] = cn[c * nvert + v];
      auto key = make_key(ids, dim);
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, c * nfc + k);
      } else {
        int64_t other = it->second;
        if (other < 0) throw std::runtime_error("face shared by more than two cells");
        int64_t f = (int64_t)fL.size();
        fL.push_back(other / nfc); fk_l.push_back((int32_t)(other % nfc));
        fR.push_back(c); fk_r.push_back(k);
        ocface[other] = f; ocside[other] = 1;
        ocface[c * nfc + k] = f; ocside[c * nfc + k] = -1;
        it->second = -1;
      }
    }
  }
  int64_t nf_int = (int64_t)fL.size();
  std::vector<int32_t> tag(nf_int, 0);
  int64_t nbound = 0;
  for (auto& kv : open) {
    if (kv.second < 0) continue;
    auto b = bmap.find(kv.first);
    if (b == bmap.end()) throw std::runtime_error("open face not listed as boundary");
    (void)b;
    ++nbound;
  }
  if (nbound != nb) throw std::runtime_error("boundary face list does not match the open faces");
  // boundary faces in order of (cell, k) for determinism
  for (int64_t c = 0; c < n; ++c)
    for (int k = 0; k < nfc; ++k) {
      if (ocface[c * nfc + k] >= 0) continue;
      int32_t ids[3];
      int m = 0;
      for (int v = 0; v < nvert; ++v) if (v != k) ids[m++] = cn[c * nvert + v];
      auto b = bmap.find(make_key(ids, dim));
      int64_t f = (int64_t)fL.size();
      fL.push_back(c); fk_l.push_back(k); fR.push_back(-1); fk_r.push_back(-1);
      tag.push_back(bft[b->second]);
      ocface[c * nfc + k] = f; ocside[c * nfc + k] = 1;
    }
  const int64_t nf = (int64_t)fL.size();
  // ---- per-face geometry (original numbering for the cells) -------------
  const int ngp = F.ngp;
  std::vector<double> fnrm(nf * dim), fS(nf), gp(nf * ngp * dim), shift(nf * dim, 0.0);
  for (int64_t f = 0; f < nf; ++f) {
    int64_t cl = fL[f];
    int kl = fk_l[f];
    double fv[3][3], fc[3] = {0, 0, 0};
    int m = 0;
    for (int v = 0; v < nvert; ++v) {
      if (v == kl) continue;
      for (int d = 0; d < dim; ++d) fv[m][d] = cx[(cl * nvert + v) * dim + d];
      ++m;
    }
    for (int v = 0; v < dim; ++v) for (int d = 0; d < dim; ++d) fc[d] += fv[v][d] / dim;
    double nn[3], S;
    if (dim == 2) {
      double ex = fv[1][0] - fv[0][0], ey = fv[1][1] - fv[0][1];
      S = std::hypot(ex, ey);
      nn[0] = ey / S; nn[1] = -ex / S;
    } else {
      double a[3], b[3];
      for (int d = 0; d < 3; ++d) { a[d] = fv[1][d] - fv[0][d]; b[d] = fv[2][d] - fv[0][d]; }
      double cr[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      double l = std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      S = 0.5 * l;
      for (int d = 0; d < 3; ++d) nn[d] = cr[d] / l;
    }
    double dot = 0.0;
    for (int d = 0; d < dim; ++d) dot += (fc[d] - cen[cl * dim + d]) * nn[d];
    if (dot < 0) for (int d = 0; d < dim; ++d) nn[d] = -nn[d];
    for (int d = 0; d < dim; ++d) fnrm[f * dim + d] = nn[d];
    fS[f] = S;
    if (dim == 2) {
      const double h = 0.5 / std::sqrt(3.0);
      for (int d = 0; d < 2; ++d) {
        gp[(f * 2 + 0) * 2 + d] = fc[d] - h * (fv[1][d] - fv[0][d]);
        gp[(f * 2 + 1) * 2 + d] = fc[d] + h * (fv[1][d] - fv[0][d]);
      }
    } else {
      for (int g = 0; g < 3; ++g)
        for (int d = 0; d < 3; ++d)
          gp[(f * 3 + g) * 3 + d] = (2.0 / 3.0) * fv[g][d] + (1.0 / 6.0) * (fv[(g + 1) % 3][d] + fv[(g + 2) % 3][d]);
    }
    int64_t cr = fR[f];
    if (cr >= 0) {
      double fcr[3] = {0, 0, 0};
      for (int v = 0; v < nvert; ++v)
        if (v != fk_r[f]) for (int d = 0; d < dim; ++d) fcr[d] += cx[(cr * nvert + v) * dim + d] / dim;
      for (int d = 0; d < dim; ++d) shift[f * dim + d] = fc[d] - fcr[d];
    }
  }
  // ---- hand over to the shared part ------------------------------------------
  FineRaw R;
  R.dim = dim; R.nfc = nfc; R.ngp = ngp; R.n = n; R.nf = nf; R.nf_int = nf_int;
  R.vol = std::move(vol); R.cen = std::move(cen); R.m2 = std::move(m2);
  R.cnf.assign(n, (int8_t)nfc);
  R.ocface = std::move(ocface); R.ocside = std::move(ocside);
  R.fL = std::move(fL); R.fR = std::move(fR); R.tag = std::move(tag);
  R.fnrm = std::move(fnrm); R.fS = std::move(fS);
  R.fngp.assign(nf, (int8_t)ngp);
  R.gw.assign(nf * ngp, 1.0 / ngp);
  R.fpt.resize(nf * dim);  // the first Gauss point lies on the (flat) face
  for (int64_t f = 0; f < nf; ++f)
    for (int d = 0; d < dim; ++d) R.fpt[f * dim + d] = gp[(f * ngp) * dim + d];
  R.gp = std::move(gp); R.shift = std::move(shift);
  finish_fine_level(R, false, F);
}


namespace {

// Faces of the mixed-element cell types in their stored order, cyclic node
// indices; -1 closes a triangle.
const int kTetF[4][4] = {{1, 2, 3, -1}, {0, 2, 3, -1}, {0, 1, 3, -1}, {0, 1, 2, -1}};
const int kPyrF[5][4] = {{0, 1, 2, 3}, {0, 1, 4, -1}, {1, 2, 4, -1}, {2, 3, 4, -1}, {3, 0, 4, -1}};
const int kPriF[5][4] = {{0, 1, 2, -1}, {3, 4, 5, -1}, {0, 1, 4, 3}, {1, 2, 5, 4}, {2, 0, 3, 5}};
const int kHexF[6][4] = {{0, 1, 2, 3}, {4, 5, 6, 7}, {0, 1, 5, 4}, {1, 2, 6, 5}, {2, 3, 7, 6}, {3, 0, 4, 7}};

int cell_faces(int type, const int (*&tab)[4]) {
  switch (type) {
    case 4: tab = kTetF; return 4;
    case 5: tab = kPyrF; return 5;
    case 6: tab = kPriF; return 5;
    case 8: tab = kHexF; return 6;
    default: tab = kTetF; return -1;
  }
}

struct QuadKey {
  std::array<int32_t, 4> v;
  bool operator==(const QuadKey& o) const { return v == o.v; }
};
struct QuadKeyHash {
  size_t operator()(const QuadKey& k) const {
    uint64_t h = 1469598103934665603ull;
    for (int i = 0; i < 4; ++i) { h ^= (uint64_t)(uint32_t)k.v[i]; h *= 1099511628211ull; }
    return (size_t)h;
  }
};
QuadKey quad_key(const int32_t* ids, int cnt) {
  QuadKey k{{-1, -1, -1, -1}};
  for (int i = 0; i < cnt; ++i) k.v[i] = ids[i];
  std::sort(k.v.begin(), k.v.begin() + cnt);
  return k;
}

inline void cross(const double* a, const double* b, double* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}

// Volume, centroid and central second moments / V of a pyramid, prism or
// hexahedron: the sum over the tetrahedra (node mean, face triangle), each
// quadrilateral face split into the 4 triangles around its node mean.  Each
// tetrahedron's second moments by the symmetric degree-2 four-point rule.
double poly_geom(int type, const double* x, double* cen, double* m2) {
  const int (*tab)[4];
  const int nfc = cell_faces(type, tab);
  const int nn = type;
  double xm[3] = {0, 0, 0};
  for (int v = 0; v < nn; ++v) for (int d = 0; d < 3; ++d) xm[d] += x[v * 3 + d] / nn;
  const double qa = 0.5854101966249685, qb = 0.1381966011250105;
  double V = 0.0, S1[3] = {0, 0, 0}, S2[9] = {0};
  auto add_tet = [&](const double* a, const double* b, const double* c) {
    // tetrahedron (0, a, b, c), coordinates about the node mean
    double cr[3];
    cross(b, c, cr);
    const double vt = std::fabs(a[0] * cr[0] + a[1] * cr[1] + a[2] * cr[2]) / 6.0;
    const double* p[4] = {nullptr, a, b, c};
    const double zero[3] = {0, 0, 0};
    p[0] = zero;
    V += vt;
    for (int q = 0; q < 4; ++q) {
      double y[3];
      for (int d = 0; d < 3; ++d) {
        double s = 0.0;
        for (int v = 0; v < 4; ++v) s += (v == q ? qa : qb) * p[v][d];
        y[d] = s;
      }
      for (int d = 0; d < 3; ++d) S1[d] += 0.25 * vt * y[d];
      for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) S2[i * 3 + j] += 0.25 * vt * y[i] * y[j];
    }
  };
  for (int k = 0; k < nfc; ++k) {
    double v[4][3];
    const int q = tab[k][3] >= 0 ? 4 : 3;
    for (int i = 0; i < q; ++i) for (int d = 0; d < 3; ++d) v[i][d] = x[tab[k][i] * 3 + d] - xm[d];
    if (q == 3) {
      add_tet(v[0], v[1], v[2]);
    } else {
      double fc[3];
      for (int d = 0; d < 3; ++d) fc[d] = 0.25 * (v[0][d] + v[1][d] + v[2][d] + v[3][d]);
      for (int i = 0; i < 4; ++i) add_tet(fc, v[i], v[(i + 1) % 4]);
    }
  }
  for (int d = 0; d < 3; ++d) cen[d] = xm[d] + S1[d] / V;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) m2[i * 3 + j] = S2[i * 3 + j] / V - (S1[i] / V) * (S1[j] / V);
  return V;
}

// Tetrahedron volume, vertex-mean centroid and second moments by the
// four-point rule (as for the simplex meshes).
double tet_geom(const double* x, double* cen, double* m2) {
  double a[3], b[3], d3[3];
  for (int k = 0; k < 3; ++k) { a[k] = x[3 + k] - x[k]; b[k] = x[6 + k] - x[k]; d3[k] = x[9 + k] - x[k]; }
  const double det = a[0] * (b[1] * d3[2] - b[2] * d3[1]) + a[1] * (b[2] * d3[0] - b[0] * d3[2]) +
                     a[2] * (b[0] * d3[1] - b[1] * d3[0]);
  for (int k = 0; k < 3; ++k) cen[k] = 0.25 * (x[k] + x[3 + k] + x[6 + k] + x[9 + k]);
  const double qa = 0.5854101966249685, qb = 0.1381966011250105;
  for (int i = 0; i < 9; ++i) m2[i] = 0.0;
  for (int q = 0; q < 4; ++q) {
    double p[3];
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int v = 0; v < 4; ++v) s += (v == q ? qa : qb) * x[v * 3 + k];
      p[k] = s - cen[k];
    }
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) m2[i * 3 + j] += 0.25 * p[i] * p[j];
  }
  return std::fabs(det) / 6.0;
}

}  // namespace

void build_fine_level_mixed(int64_t n, const int32_t* type, const int64_t* off, const int32_t* cn, const double* cx,
                            int64_t nb, const int64_t* boff, const int32_t* bfn, const int32_t* bft, FineLevel& F) {
  if (n <= 0) throw std::runtime_error("mesh has no cells");
  const int dim = 3, nfc = 6, ngp = 4;
  FineRaw R;
  R.dim = dim; R.nfc = nfc; R.ngp = ngp; R.n = n;
  R.vol.resize(n); R.cen.resize(n * 3); R.m2.resize(n * 9); R.cnf.resize(n);
  for (int64_t c = 0; c < n; ++c) {
    const int (*tab)[4];
    const int nf = cell_faces(type[c], tab);
    if (nf < 0 || off[c + 1] - off[c] != type[c])
      throw std::runtime_error("cell " + std::to_string(c) + ": unknown type or node count");
    R.cnf[c] = (int8_t)nf;
    const double* x = cx + off[c] * 3;
    R.vol[c] = type[c] == 4 ? tet_geom(x, &R.cen[c * 3], &R.m2[c * 9]) : poly_geom(type[c], x, &R.cen[c * 3], &R.m2[c * 9]);
    if (!(R.vol[c] > 0.0)) throw std::runtime_error("degenerate cell " + std::to_string(c));
  }
  // ---- faces ----------------------------------------------------------
  std::unordered_map<QuadKey, int64_t, QuadKeyHash> bmap;
  bmap.reserve(nb * 2 + 1);
  for (int64_t b = 0; b < nb; ++b) {
    const int q = (int)(boff[b + 1] - boff[b]);
    if (q != 3 && q != 4) throw std::runtime_error("boundary face with " + std::to_string(q) + " nodes");
    if (!bmap.emplace(quad_key(bfn + boff[b], q), b).second) throw std::runtime_error("duplicate boundary face");
  }
  std::unordered_map<QuadKey, int64_t, QuadKeyHash> open;  // key -> cell*nfc + k
  open.reserve(n * nfc);
  R.ocface.assign(n * nfc, -1);
  R.ocside.assign(n * nfc, 0);
  std::vector<int32_t> fk_l;
  auto face_ids = [&](int64_t c, int k, int32_t* ids) {
    const int (*tab)[4];
    cell_faces(type[c], tab);
    const int q = tab[k][3] >= 0 ? 4 : 3;
    for (int i = 0; i < q; ++i) ids[i] = cn[off[c] + tab[k][i]];
    return q;
  };
  for (int64_t c = 0; c < n; ++c)
    for (int k = 0; k < R.cnf[c]; ++k) {
      int32_t ids[4];
      const int q = face_ids(c, k, ids);
      auto key = quad_key(ids, q);
      auto it = open.find(key);
      if (it == open.end()) {
        open.emplace(key, c * nfc + k);
      } else {
        const int64_t other = it->second;
        if (other < 0) throw std::runtime_error("face shared by more than two cells");
        const int64_t f = (int64_t)R.fL.size();
        R.fL.push_back(other / nfc); fk_l.push_back((int32_t)(other % nfc));
        R.fR.push_back(c);
        R.ocface[other] = f; R.ocside[other] = 1;
        R.ocface[c * nfc + k] = f; R.ocside[c * nfc + k] = -1;
        it->second = -1;
      }
    }
  R.nf_int = (int64_t)R.fL.size();
  R.tag.assign(R.nf_int, 0);
  int64_t nbound = 0;
  for (auto& kv : open)
    if (kv.second >= 0) {
      if (bmap.find(kv.first) == bmap.end()) throw std::runtime_error("open face not listed as boundary");
      ++nbound;
    }
  if (nbound != nb) throw std::runtime_error("boundary face list does not match the open faces");
  for (int64_t c = 0; c < n; ++c)
    for (int k = 0; k < R.cnf[c]; ++k) {
      if (R.ocface[c * nfc + k] >= 0) continue;
      int32_t ids[4];
      const int q = face_ids(c, k, ids);
      auto b = bmap.find(quad_key(ids, q));
      const int64_t f = (int64_t)R.fL.size();
      R.fL.push_back(c); fk_l.push_back(k); R.fR.push_back(-1);
      R.tag.push_back(bft[b->second]);
      R.ocface[c * nfc + k] = f; R.ocside[c * nfc + k] = 1;
    }
  const int64_t nf = (int64_t)R.fL.size();
  R.nf = nf;
  // ---- per-face geometry from the owning (L) cell's cyclic vertices --------
  // triangle: area vector 1/2 (v1 - v0) x (v2 - v0), the degree-2 rule of the
  // simplex meshes (barycentric 2/3, 1/6, 1/6), equal weights; quadrilateral
  // (Sec 2.2, four Gauss points): area vector 1/2 (v2 - v0) x (v3 - v1), the
  // 2 x 2 Gauss-Legendre points of the bilinear surface sum N_i(s, t) v_i,
  // weights proportional to |x_s x x_t| there.  Normals point out of L; the
  // ghost mirror plane passes through the face's node mean.
  R.fnrm.assign(nf * 3, 0.0); R.fS.assign(nf, 0.0); R.fngp.assign(nf, 0);
  R.gp.assign(nf * ngp * 3, 0.0); R.gw.assign(nf * ngp, 0.0);
  R.shift.assign(nf * 3, 0.0); R.fpt.assign(nf * 3, 0.0);
  const double r3 = 1.0 / std::sqrt(3.0);
  for (int64_t f = 0; f < nf; ++f) {
    const int64_t cl = R.fL[f];
    const int (*tab)[4];
    cell_faces(type[cl], tab);
    const int kl = fk_l[f];
    const int q = tab[kl][3] >= 0 ? 4 : 3;
    double v[4][3], fc[3] = {0, 0, 0};
    for (int i = 0; i < q; ++i)
      for (int d = 0; d < 3; ++d) {
        v[i][d] = cx[(off[cl] + tab[kl][i]) * 3 + d];
        fc[d] += v[i][d] / q;
      }
    double a[3], b[3], A[3];
    for (int d = 0; d < 3; ++d) {
      a[d] = q == 3 ? v[1][d] - v[0][d] : v[2][d] - v[0][d];
      b[d] = q == 3 ? v[2][d] - v[0][d] : v[3][d] - v[1][d];
    }
    cross(a, b, A);
    const double l = std::sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    double nn[3] = {A[0] / l, A[1] / l, A[2] / l};
    double dot = 0.0;
    for (int d = 0; d < 3; ++d) dot += (fc[d] - R.cen[cl * 3 + d]) * nn[d];
    if (dot < 0) for (int d = 0; d < 3; ++d) nn[d] = -nn[d];
    for (int d = 0; d < 3; ++d) { R.fnrm[f * 3 + d] = nn[d]; R.fpt[f * 3 + d] = fc[d]; }
    R.fS[f] = 0.5 * l;
    R.fngp[f] = (int8_t)(q == 4 ? 4 : 3);
    if (q == 3) {
      for (int g = 0; g < 3; ++g) {
        for (int d = 0; d < 3; ++d)
          R.gp[(f * ngp + g) * 3 + d] = (2.0 / 3.0) * v[g][d] + (1.0 / 6.0) * (v[(g + 1) % 3][d] + v[(g + 2) % 3][d]);
        R.gw[f * ngp + g] = 1.0 / 3.0;
      }
      continue;
    }
    const double ss[4] = {-r3, r3, r3, -r3}, tt[4] = {-r3, -r3, r3, r3};
    double wsum = 0.0, wj[4];
    for (int g = 0; g < 4; ++g) {
      const double s = ss[g], t = tt[g];
      const double N[4] = {(1 - s) * (1 - t) / 4, (1 + s) * (1 - t) / 4, (1 + s) * (1 + t) / 4, (1 - s) * (1 + t) / 4};
      const double Ns[4] = {-(1 - t) / 4, (1 - t) / 4, (1 + t) / 4, -(1 + t) / 4};
      const double Nt[4] = {-(1 - s) / 4, -(1 + s) / 4, (1 + s) / 4, (1 - s) / 4};
      double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
      for (int d = 0; d < 3; ++d) {
        double p = 0.0;
        for (int i = 0; i < 4; ++i) { p += N[i] * v[i][d]; xs[d] += Ns[i] * v[i][d]; xt[d] += Nt[i] * v[i][d]; }
        R.gp[(f * ngp + g) * 3 + d] = p;
      }
      double j3[3];
      cross(xs, xt, j3);
      wj[g] = std::sqrt(j3[0] * j3[0] + j3[1] * j3[1] + j3[2] * j3[2]);
      wsum += wj[g];
    }
    for (int g = 0; g < 4; ++g) R.gw[f * ngp + g] = wj[g] / wsum;
  }
  finish_fine_level(R, true, F);
}

void build_coarse_level(const Hierarchy& H, int li, const int32_t* parent_orig, CoarseLevel& C) {
  // previous level view (new ids)
  const bool from_fine = li == 0;
  const FineLevel& Fn = H.fine;
  const CoarseLevel* Pc = from_fine ? nullptr : &H.coarse[li - 1];
  const int dim = Fn.dim;
  const int64_t np = from_fine ? Fn.n : Pc->n;
  const std::vector<int64_t>& piperm = from_fine ? Fn.iperm : Pc->iperm;
  const std::vector<int64_t>& pfL = from_fine ? Fn.fL : Pc->fL;
  const std::vector<int64_t>& pfR = from_fine ? Fn.fR : Pc->fR;
  const std::vector<int32_t>& pftag = from_fine ? Fn.ftag : Pc->ftag;
  const std::vector<double>& pfn = from_fine ? Fn.fn : Pc->fn;
  const std::vector<double>& pfS = from_fine ? Fn.fS : Pc->fS;
  const std::vector<double>& pvol = from_fine ? Fn.vol : Pc->vol;
  const std::vector<double>& pcen = from_fine ? Fn.cen : Pc->cen;
  int64_t nc = 0;
  for (int64_t i = 0; i < np; ++i) {
    if (parent_orig[i] < 0) throw std::runtime_error("negative parent id");
    nc = std::max<int64_t>(nc, (int64_t)parent_orig[i] + 1);
  }
  // parent of each previous-level cell (new id) in coarse ORIGINAL ids
  std::vector<int64_t> par(np);
  for (int64_t i = 0; i < np; ++i) par[i] = parent_orig[piperm[i]];
  // coarse faces keyed by (I, J) (I < J, original ids) or (I, -1 - tag)
  struct Acc { double sn[3]; };
  std::vector<std::pair<std::pair<int64_t, int64_t>, Acc>> rec;
  rec.reserve(pfL.size());
  for (size_t f = 0; f < pfL.size(); ++f) {
    int64_t I = par[pfL[f]];
    Acc a{{0, 0, 0}};
    if (pfR[f] < 0) {
      for (int d = 0; d < dim; ++d) a.sn[d] = pfS[f] * pfn[f * dim + d];
      rec.push_back({{I, -1 - (int64_t)pftag[f]}, a});
      continue;
    }
    int64_t J = par[pfR[f]];
    if (I == J) continue;
    double sg = I < J ? 1.0 : -1.0;
    for (int d = 0; d < dim; ++d) a.sn[d] = sg * pfS[f] * pfn[f * dim + d];
    rec.push_back({{std::min(I, J), std::max(I, J)}, a});
  }
  std::stable_sort(rec.begin(), rec.end(), [](const auto& x, const auto& y) {
    // interior pairs sorted by (I, J); boundary entries (J < 0) after all
    // interior neighbours of I, by tag
    if (x.first.first != y.first.first) return x.first.first < y.first.first;
    bool xb = x.first.second < 0, yb = y.first.second < 0;
    if (xb != yb) return !xb;
    if (!xb) return x.first.second < y.first.second;
    return x.first.second > y.first.second;  // -1-tag descending = tag ascending
  });
  std::vector<int64_t> cI, cJ;
  std::vector<int32_t> ctag;
  std::vector<double> csn;
  for (size_t i = 0; i < rec.size();) {
    size_t j = i;
    double s[3] = {0, 0, 0};
    while (j < rec.size() && rec[j].first == rec[i].first) {
      for (int d = 0; d < dim; ++d) s[d] += rec[j].second.sn[d];
      ++j;
    }
    cI.push_back(rec[i].first.first);
    int64_t J = rec[i].first.second;
    cJ.push_back(J >= 0 ? J : -1);
    ctag.push_back(J >= 0 ? 0 : (int32_t)(-1 - J));
    for (int d = 0; d < dim; ++d) csn.push_back(s[d]);
    i = j;
  }
  const int64_t nf = (int64_t)cI.size();
  // per-cell face lists in (neighbour original id, tag) order
  std::vector<std::vector<std::pair<std::pair<int64_t, int32_t>, int64_t>>> lists(nc);
  for (int64_t f = 0; f < nf; ++f) {
    lists[cI[f]].push_back({{cJ[f] >= 0 ? cJ[f] : INT64_MAX, ctag[f]}, f});
    if (cJ[f] >= 0) lists[cJ[f]].push_back({{cI[f], 0}, f});
  }
  std::vector<int64_t> off(nc + 1, 0), nbr;
  for (int64_t I = 0; I < nc; ++I) {
    std::sort(lists[I].begin(), lists[I].end());
    off[I + 1] = off[I] + (int64_t)lists[I].size();
    for (auto& e : lists[I]) {
      int64_t f = e.second;
      nbr.push_back(cI[f] == I ? cJ[f] : cI[f]);
    }
  }
  C.n = nc;
  C.n_colors = greedy_colouring(nc, off, nbr, C.color_orig);
  renumber(C.color_orig, C.n_colors, C.perm, C.iperm, C.color_off);
  // geometry
  C.vol.assign(nc, 0.0);
  C.cen.assign(nc * dim, 0.0);
  std::vector<double> vo(nc, 0.0), co(nc * dim, 0.0);
  for (int64_t i = 0; i < np; ++i) {
    vo[par[i]] += pvol[i];
    for (int d = 0; d < dim; ++d) co[par[i] * dim + d] += pvol[i] * pcen[i * dim + d];
  }
  for (int64_t I = 0; I < nc; ++I) {
    if (!(vo[I] > 0.0)) throw std::runtime_error("coarse cell without children");
    int64_t J = C.perm[I];
    C.vol[J] = vo[I];
    for (int d = 0; d < dim; ++d) C.cen[J * dim + d] = co[I * dim + d] / vo[I];
  }
  // faces in new ids
  C.nf = nf;
  C.fL.resize(nf); C.fR.resize(nf); C.ftag = ctag; C.fn.resize(nf * dim); C.fS.resize(nf);
  for (int64_t f = 0; f < nf; ++f) {
    C.fL[f] = C.perm[cI[f]];
    C.fR[f] = cJ[f] >= 0 ? C.perm[cJ[f]] : -1;
    double S = 0.0;
    for (int d = 0; d < dim; ++d) S += csn[f * dim + d] * csn[f * dim + d];
    S = std::sqrt(S);
    C.fS[f] = S;
    for (int d = 0; d < dim; ++d) C.fn[f * dim + d] = csn[f * dim + d] / S;
  }
  // cell -> face CSR in new order
  C.cf_off.assign(nc + 1, 0);
  for (int64_t J = 0; J < nc; ++J) C.cf_off[J + 1] = C.cf_off[J] + (int64_t)lists[C.iperm[J]].size();
  C.cf_face.resize(C.cf_off[nc]);
  C.cf_side.resize(C.cf_off[nc]);
  for (int64_t J = 0; J < nc; ++J) {
    int64_t I = C.iperm[J];
    int64_t e = C.cf_off[J];
    for (auto& it : lists[I]) {
      int64_t f = it.second;
      C.cf_face[e] = f;
      C.cf_side[e] = cI[f] == I ? 1 : -1;
      ++e;
    }
  }
  // children and parents (new ids)
  C.parent_of_fine.resize(np);
  for (int64_t i = 0; i < np; ++i) C.parent_of_fine[i] = C.perm[par[i]];
  C.ch_off.assign(nc + 1, 0);
  for (int64_t i = 0; i < np; ++i) C.ch_off[C.parent_of_fine[i] + 1]++;
  for (int64_t J = 0; J < nc; ++J) C.ch_off[J + 1] += C.ch_off[J];
  C.ch_idx.resize(np);
  std::vector<int64_t> pos(C.ch_off.begin(), C.ch_off.end() - 1);
  for (int64_t i = 0; i < np; ++i) C.ch_idx[pos[C.parent_of_fine[i]]++] = i;
}

}  // namespace cgks
