// Agglomeration coarsening by hash-selected face removal with a skewness guard
// (Sec 5.1, Eqs. hash value, virtual center, skewness factor; Algorithm
// cell-merge), for hierarchies of meshes that are not nested by construction.
//
// Readings (the paper leaves them open):
//  * interior faces are visited in the order of their (lower, higher) cell-id
//    pair, N_l = lower id, N_r = higher id, N_f = number of interior faces;
//    the hash is h = [23 (N_l + N_r) + N_l N_r] mod N_f as printed (the
//    paper's worked example, h = 5 for ids 10, 12 and N_f = 100, does not
//    follow from it: the formula gives 26);
//  * a face enters the collection when its hash is new; faces of the
//    collection are then visited in the same order and merge their two cells
//    when neither cell has been merged in this pass (pairwise merging, so a
//    pass at most halves the cell count) and the skewness test passes;
//  * the skewness of Eq. skewness factor is taken for every face of the merged
//    cell other than the removed one, with d from the virtual center of
//    Eq. virtual center to the face center and n the outward unit normal;
//    the merge happens when the smallest sin(alpha) = d.n / |d| is above the
//    limit (a face with d = 0 counts as sin(alpha) = -1);
//  * boundary faces are never removed (the paper keeps them), nor faces on a
//    periodic seam (seen at different positions from its two cells), which
//    play the role of the paper's parallel interfaces;
//  * the faces of a level, the fine one included, are its neighbour pairs
//    (the union of the fine faces between two cells) and the union of a
//    cell's boundary faces with one tag: area vectors summed, centers
//    weighted by fine face area, a pair on a periodic seam if any of its fine
//    faces is; interior faces in (lower id, higher id) order;
//  * coarse ids follow the lowest member id;
//  * one level applies `passes` such passes, each on the graph of the
//    previous pass's agglomerates (2 passes give about 4:1 in 2D, 3 about
//    8:1 in 3D, the ratios of nested refinement).
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <stdexcept>
#include <vector>

#include "host_mesh.hpp"

namespace cgks {
namespace {

struct GFace {
  int64_t L = -1, R = -1;   // R = -1: boundary
  double a[3] = {0, 0, 0};  // area vector, out of L
  double cl[3] = {0, 0, 0}; // center as seen from L's frame
  double cr[3] = {0, 0, 0}; // center as seen from R's frame
  double area = 0;          // |a|
  double w = 0;             // sum of the fine face areas (weights of the centers)
  int32_t tag = 0;          // boundary tag (boundary faces)
  bool seam = false;        // periodic seam: never removed
};

struct Graph {
  int dim = 0;
  int64_t n = 0;
  std::vector<double> vol, cen;  // [n], [n][dim] (each cell in its own frame)
  std::vector<GFace> faces;      // interior faces first, in (L, R) order, then boundary faces
  int64_t nf_int = 0;
};

double simplex_volume(int dim, const double* x) {
  if (dim == 2) {
    return 0.5 * std::fabs((x[2] - x[0]) * (x[5] - x[1]) - (x[4] - x[0]) * (x[3] - x[1]));
  }
  double e[3][3];
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) e[i][d] = x[(i + 1) * 3 + d] - x[d];
  const double det = e[0][0] * (e[1][1] * e[2][2] - e[1][2] * e[2][1]) -
                     e[0][1] * (e[1][0] * e[2][2] - e[1][2] * e[2][0]) +
                     e[0][2] * (e[1][0] * e[2][1] - e[1][1] * e[2][0]);
  return std::fabs(det) / 6.0;
}

// face opposite vertex k of a simplex: center, area vector pointing away from vertex k
void simplex_face(int dim, const double* x, int k, double* c, double* a) {
  int v[3], m = 0;
  for (int i = 0; i <= dim; ++i)
    if (i != k) v[m++] = i;
  for (int d = 0; d < dim; ++d) {
    double s = 0;
    for (int i = 0; i < dim; ++i) s += x[v[i] * dim + d];
    c[d] = s / dim;
  }
  if (dim == 2) {
    const double tx = x[v[1] * 2] - x[v[0] * 2], ty = x[v[1] * 2 + 1] - x[v[0] * 2 + 1];
    a[0] = ty;
    a[1] = -tx;
  } else {
    double u[3], w[3];
    for (int d = 0; d < 3; ++d) {
      u[d] = x[v[1] * 3 + d] - x[v[0] * 3 + d];
      w[d] = x[v[2] * 3 + d] - x[v[0] * 3 + d];
    }
    a[0] = 0.5 * (u[1] * w[2] - u[2] * w[1]);
    a[1] = 0.5 * (u[2] * w[0] - u[0] * w[2]);
    a[2] = 0.5 * (u[0] * w[1] - u[1] * w[0]);
  }
  // orient away from vertex k
  double s = 0;
  for (int d = 0; d < dim; ++d) s += a[d] * (c[d] - x[k * dim + d]);
  if (s < 0)
    for (int d = 0; d < dim; ++d) a[d] = -a[d];
}

Graph fine_graph(int dim, int64_t n, const int32_t* cn, const double* cx, int64_t nb, const int32_t* bn,
                 const int32_t* bt) {
  Graph G;
  G.dim = dim;
  G.n = n;
  G.vol.resize(n);
  G.cen.assign((size_t)n * dim, 0.0);
  const int nv = dim + 1;
  for (int64_t c = 0; c < n; ++c) {
    const double* x = cx + (size_t)c * nv * dim;
    G.vol[c] = simplex_volume(dim, x);
    for (int d = 0; d < dim; ++d) {
      double s = 0;
      for (int i = 0; i < nv; ++i) s += x[i * dim + d];
      G.cen[(size_t)c * dim + d] = s / nv;
    }
  }
  // match faces by their sorted node ids
  std::map<std::array<int32_t, 3>, std::vector<std::pair<int64_t, int>>> owners;
  for (int64_t c = 0; c < n; ++c)
    for (int k = 0; k < nv; ++k) {
      std::array<int32_t, 3> key = {-1, -1, -1};
      int m = 0;
      for (int i = 0; i < nv; ++i)
        if (i != k) key[m++] = cn[(size_t)c * nv + i];
      std::sort(key.begin(), key.begin() + dim);
      owners[key].push_back({c, k});
    }
  std::map<std::array<int32_t, 3>, int> bset;
  for (int64_t b = 0; b < nb; ++b) {
    std::array<int32_t, 3> key = {-1, -1, -1};
    for (int i = 0; i < dim; ++i) key[i] = bn[(size_t)b * dim + i];
    std::sort(key.begin(), key.begin() + dim);
    bset[key] = bt[b];
  }
  std::vector<GFace> inner, bnd;
  for (const auto& kv : owners) {
    const auto& o = kv.second;
    if (o.size() == 2) {
      int64_t L = o[0].first, R = o[1].first;
      int kl = o[0].second, kr = o[1].second;
      if (L > R) {
        std::swap(L, R);
        std::swap(kl, kr);
      }
      GFace f;
      f.L = L;
      f.R = R;
      double ar[3];
      simplex_face(dim, cx + (size_t)L * nv * dim, kl, f.cl, f.a);
      simplex_face(dim, cx + (size_t)R * nv * dim, kr, f.cr, ar);
      double s2 = 0, sc = 0;
      for (int d = 0; d < dim; ++d) {
        s2 += f.a[d] * f.a[d];
        sc += (f.cl[d] - f.cr[d]) * (f.cl[d] - f.cr[d]);
      }
      f.area = f.w = std::sqrt(s2);
      // seen at two positions (a periodic image) unless they agree to 1e-6 of the face size
      const double h2 = dim == 2 ? s2 : f.area;
      f.seam = sc > 1e-12 * h2;
      inner.push_back(f);
    } else if (o.size() == 1) {
      auto it = bset.find(kv.first);
      if (it == bset.end()) throw std::runtime_error("agglomeration: open face without a boundary tag");
      GFace f;
      f.L = o[0].first;
      f.tag = it->second;
      simplex_face(dim, cx + (size_t)f.L * nv * dim, o[0].second, f.cl, f.a);
      double s2 = 0;
      for (int d = 0; d < dim; ++d) s2 += f.a[d] * f.a[d];
      f.area = f.w = std::sqrt(s2);
      for (int d = 0; d < dim; ++d) f.cr[d] = f.cl[d];
      bnd.push_back(f);
    } else {
      throw std::runtime_error("agglomeration: non-manifold face");
    }
  }
  std::sort(inner.begin(), inner.end(),
            [](const GFace& a, const GFace& b) { return a.L != b.L ? a.L < b.L : a.R < b.R; });
  std::stable_sort(bnd.begin(), bnd.end(),
                   [](const GFace& a, const GFace& b) { return a.L != b.L ? a.L < b.L : a.tag < b.tag; });
  G.nf_int = (int64_t)inner.size();
  G.faces = inner;
  G.faces.insert(G.faces.end(), bnd.begin(), bnd.end());
  return G;
}

// one pass: parent of every cell of G (coarse ids by lowest member)
std::vector<int32_t> merge_pass(const Graph& G, double min_skew) {
  const int dim = G.dim;
  const int64_t n = G.n, nfi = G.nf_int;
  // faces of each cell
  std::vector<std::vector<int64_t>> cf(n);
  for (int64_t f = 0; f < (int64_t)G.faces.size(); ++f) {
    cf[G.faces[f].L].push_back(f);
    if (G.faces[f].R >= 0) cf[G.faces[f].R].push_back(f);
  }
  // 1. collection of faces with a new hash value (Eq. hash value)
  std::vector<int64_t> coll;
  if (nfi > 0) {
    std::vector<char> seen((size_t)nfi, 0);
    for (int64_t f = 0; f < nfi; ++f) {
      const int64_t l = G.faces[f].L, r = G.faces[f].R;
      const int64_t h = (23 * (l + r) + l * r) % nfi;
      if (!seen[h]) {
        seen[h] = 1;
        coll.push_back(f);
      }
    }
  }
  // 2. merge pairs that pass the skewness test
  std::vector<int64_t> partner(n, -1);
  for (int64_t f : coll) {
    const GFace& F = G.faces[f];
    const int64_t l = F.L, r = F.R;
    if (F.seam || partner[l] >= 0 || partner[r] >= 0) continue;
    // r's centroid in l's frame (the shared face is not a seam: same frame)
    double C[3];
    const double vl = G.vol[l], vr = G.vol[r];
    for (int d = 0; d < dim; ++d)
      C[d] = (vl * G.cen[(size_t)l * dim + d] + vr * G.cen[(size_t)r * dim + d]) / (vl + vr);
    double smin = 2.0;
    for (int side = 0; side < 2; ++side) {
      const int64_t c = side == 0 ? l : r;
      for (int64_t g : cf[c]) {
        const GFace& H = G.faces[g];
        const int64_t other = H.L == c ? H.R : H.L;
        if (other == (side == 0 ? r : l)) continue;  // the removed face
        const bool out_of_L = H.L == c;
        const double* xc = out_of_L ? H.cl : H.cr;
        double dd[3], s = 0, dn = 0;
        for (int d = 0; d < dim; ++d) {
          dd[d] = xc[d] - C[d];
          dn += dd[d] * dd[d];
          s += dd[d] * (out_of_L ? H.a[d] : -H.a[d]);
        }
        const double sa = dn > 0.0 ? s / (std::sqrt(dn) * H.area) : -1.0;
        smin = std::min(smin, sa);
      }
    }
    if (smin > min_skew) {
      partner[l] = r;
      partner[r] = l;
    }
  }
  std::vector<int32_t> parent(n, -1);
  int32_t k = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (parent[c] >= 0) continue;
    parent[c] = k;
    if (partner[c] >= 0) parent[partner[c]] = k;
    ++k;
  }
  return parent;
}

Graph coarse_graph(const Graph& G, const std::vector<int32_t>& parent) {
  const int dim = G.dim;
  Graph C;
  C.dim = dim;
  C.n = *std::max_element(parent.begin(), parent.end()) + 1;
  C.vol.assign(C.n, 0.0);
  C.cen.assign((size_t)C.n * dim, 0.0);
  for (int64_t c = 0; c < G.n; ++c) {
    C.vol[parent[c]] += G.vol[c];
    for (int d = 0; d < dim; ++d) C.cen[(size_t)parent[c] * dim + d] += G.vol[c] * G.cen[(size_t)c * dim + d];
  }
  for (int64_t c = 0; c < C.n; ++c)
    for (int d = 0; d < dim; ++d) C.cen[(size_t)c * dim + d] /= C.vol[c];
  std::map<std::pair<int64_t, int64_t>, GFace> inner, bnd;
  for (const GFace& F : G.faces) {
    const int64_t A = parent[F.L];
    if (F.R < 0) {
      GFace& b = bnd[{A, (int64_t)F.tag}];
      b.L = A;
      b.tag = F.tag;
      for (int d = 0; d < dim; ++d) {
        b.a[d] += F.a[d];
        b.cl[d] += F.w * F.cl[d];
      }
      b.w += F.w;
      continue;
    }
    const int64_t B = parent[F.R];
    if (A == B) continue;
    const bool keep = A < B;  // orientation from the lower coarse id
    const int64_t lo = keep ? A : B, hi = keep ? B : A;
    GFace& H = inner[{lo, hi}];
    H.L = lo;
    H.R = hi;
    for (int d = 0; d < dim; ++d) {
      H.a[d] += keep ? F.a[d] : -F.a[d];
      H.cl[d] += F.w * (keep ? F.cl[d] : F.cr[d]);
      H.cr[d] += F.w * (keep ? F.cr[d] : F.cl[d]);
    }
    H.w += F.w;
    H.seam = H.seam || F.seam;
  }
  for (auto& kv : inner) {
    GFace f = kv.second;
    double s2 = 0;
    for (int d = 0; d < dim; ++d) {
      f.cl[d] /= f.w;
      f.cr[d] /= f.w;
      s2 += f.a[d] * f.a[d];
    }
    f.area = std::sqrt(s2);
    C.faces.push_back(f);
  }
  C.nf_int = (int64_t)C.faces.size();
  for (auto& kv : bnd) {
    GFace f = kv.second;
    double s2 = 0;
    for (int d = 0; d < dim; ++d) {
      f.cl[d] /= f.w;
      f.cr[d] = f.cl[d];
      s2 += f.a[d] * f.a[d];
    }
    f.area = std::sqrt(s2);
    C.faces.push_back(f);
  }
  return C;
}

}  // namespace

void agglomerate(int dim, int64_t n, const int32_t* cell_nodes, const double* cell_xyz, int64_t nb,
                 const int32_t* bface_nodes, const int32_t* bface_tag, int n_levels, int passes,
                 double min_skew, std::vector<std::vector<int32_t>>& parents) {
  parents.clear();
  // the faces of every level are its neighbour pairs and its (cell, tag)
  // boundary groups, as on the coarse levels of the solver
  std::vector<int32_t> id(n);
  for (int64_t c = 0; c < n; ++c) id[c] = (int32_t)c;
  Graph G = coarse_graph(fine_graph(dim, n, cell_nodes, cell_xyz, nb, bface_nodes, bface_tag), id);
  for (int l = 1; l < n_levels; ++l) {
    std::vector<int32_t> p(G.n);
    for (int64_t c = 0; c < G.n; ++c) p[c] = (int32_t)c;
    for (int k = 0; k < passes; ++k) {
      std::vector<int32_t> q = merge_pass(G, min_skew);
      for (auto& v : p) v = q[v];
      G = coarse_graph(G, q);
    }
    parents.push_back(std::move(p));
  }
}

}  // namespace cgks
