// Host-side mesh preprocessing for the CGKS library: faces, geometry, the
// per-cell constrained least-squares reconstruction operator, colouring and
// colour-major renumbering, and the agglomerated coarse levels.
//
// Paper (arXiv 2509.06347) sections: Sec 2.2 (finite volumes, face Gauss
// points), Sec 3.1-3.2 (reconstruction stencils), Sec 4.1 (colouring),
// Sec 5.1 (coarse-cell geometry).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace cgks {

constexpr int kMaxDim = 3;
constexpr int kMaxVar = 5;

// Fine level (simplices, or 3-D mixed elements).  All arrays are in the
// colour-major cell order ("new" ids); iperm maps new -> original.
struct FineLevel {
  int dim = 0, nv = 0, ngp = 0, nfc = 0;  // simplices: nfc = dim + 1 faces per cell, ngp points per face;
                                           // mixed elements: the maxima 6 and 4 (arrays padded to them)
  bool mixed = false;
  std::vector<int8_t> cnf;           // [n] faces of each cell (mixed elements only)
  std::vector<int8_t> fngp;          // [nf] Gauss points of each face (mixed elements only)
  std::vector<double> gw;            // [nf][ngp] their weights, summing to 1 (mixed elements only)
  int nk = 0;                              // quadratic basis size (5 / 9)
  int64_t n = 0;
  int n_colors = 0;
  std::vector<int32_t> color_orig;   // colour of each original cell (1..Nc)
  std::vector<int64_t> perm, iperm;  // original -> new, new -> original
  std::vector<int64_t> color_off;    // [Nc + 1] colour ranges in new order
  std::vector<double> vol;           // [n]
  std::vector<double> cen;           // [n][dim]
  std::vector<double> m2;            // [n][dim*dim] central second moments / V
  // faces: interior first, then boundary
  int64_t nf = 0, nf_int = 0;
  std::vector<int64_t> fL, fR;       // R = -1 on boundary faces
  std::vector<int32_t> ftag;
  std::vector<double> fn, fS;        // [nf][dim], [nf]
  std::vector<double> XL, XR;        // [nf][ngp][dim] Gauss point minus L / R centroid
  // cell -> faces in stored order (face k opposite vertex k)
  std::vector<int64_t> cface;        // [n][nfc]
  std::vector<int8_t> cside;         // +1 if the cell is the face's L
  std::vector<int64_t> cnbr;         // [n][nfc] neighbour (new id) or -1
  // reconstruction: a = OpE e + OpD d (per variable), e_m = Q_m - Q_0,
  // d_{m,d} = neighbour slope; avg0 = <X^k>_0 so that c0 = Q_0 - a . avg0
  int nop = 0;                       // nk * (nfc + nfc*dim)
  std::vector<double> op;            // [n][nk][nfc + nfc*dim]
  std::vector<int8_t> op_ok;         // 0 if the stencil is degenerate (p1 only)
  std::vector<double> avg0;          // [n][nk]
  std::vector<double> gg;            // [n][nfc][dim]  S_m n_m / (2 V_0) outward
};

// Agglomerated coarse level.
struct CoarseLevel {
  int64_t n = 0;
  int n_colors = 0;
  std::vector<int32_t> color_orig;
  std::vector<int64_t> perm, iperm, color_off;
  std::vector<double> vol;
  std::vector<double> cen;
  // faces (unique neighbour pairs / boundary (cell, tag)); new ids
  int64_t nf = 0;
  std::vector<int64_t> fL, fR;
  std::vector<int32_t> ftag;
  std::vector<double> fn, fS;
  // cell -> faces CSR in new order, sorted by (original neighbour id, tag)
  std::vector<int64_t> cf_off, cf_face;
  std::vector<int8_t> cf_side;
  // children (previous level, new ids) CSR, and parent of each child
  std::vector<int64_t> ch_off, ch_idx;
  std::vector<int64_t> parent_of_fine;  // [n_prev] previous-level new id -> this level new id
};

struct Hierarchy {
  FineLevel fine;
  std::vector<CoarseLevel> coarse;
};

// Builds the fine level.  cell_nodes [n][dim+1], cell_xyz [n][dim+1][dim],
// bface_nodes [nb][dim], bface_tag [nb].  Throws std::runtime_error.
void build_fine_level(int dim, int64_t n, const int32_t* cell_nodes, const double* cell_xyz,
                      int64_t nb, const int32_t* bface_nodes, const int32_t* bface_tag,
                      FineLevel& out);

// Builds the fine level of a 3-D mesh of tetrahedra, pyramids, prisms and
// hexahedra: cell_type [n] = node count (4, 5, 6, 8), cell_node_off [n+1],
// cell_nodes and cell_xyz [sum][3] in each type's node order (pyramid: base
// 0-1-2-3 cyclic, apex 4; prism: triangles 0-1-2 and 3-4-5, 3 above 0;
// hexahedron: 0-1-2-3 and 4-5-6-7 cyclic, 4 above 0); boundary faces by
// bface_node_off [nb+1], bface_nodes (3 or 4 ids), bface_tag [nb].
void build_fine_level_mixed(int64_t n, const int32_t* cell_type, const int64_t* cell_node_off,
                            const int32_t* cell_nodes, const double* cell_xyz, int64_t nb,
                            const int64_t* bface_node_off, const int32_t* bface_nodes, const int32_t* bface_tag,
                            FineLevel& out);

// Adds a coarse level below `prev_*` (parent given in the previous level's
// ORIGINAL numbering -> coarse original ids).
void build_coarse_level(const Hierarchy& H, int level_index, const int32_t* parent_orig,
                        CoarseLevel& out);

// Agglomeration coarsening by hash-selected face removal with a skewness
// guard (Sec 5.1).  Same mesh arrays as build_fine_level, original order.
// parents[l-1][i] = level-l agglomerate of level-(l-1) cell i, for
// l = 1..n_levels-1; each level is `passes` pairwise merge passes; a merge
// needs every remaining face of the merged cell to have sin(alpha) > min_skew.
// Throws std::runtime_error for a mesh that build_fine_level would reject.
void agglomerate(int dim, int64_t n, const int32_t* cell_nodes, const double* cell_xyz, int64_t nb,
                 const int32_t* bface_nodes, const int32_t* bface_tag, int n_levels, int passes,
                 double min_skew, std::vector<std::vector<int32_t>>& parents);

// Breadth-first greedy colouring from cell 0 (Sec 4.1).  nbr lists per cell
// in stored order (-1 = no neighbour).  Returns number of colours.
int greedy_colouring(int64_t n, const std::vector<int64_t>& off, const std::vector<int64_t>& nbr,
                     std::vector<int32_t>& colour);

}  // namespace cgks
