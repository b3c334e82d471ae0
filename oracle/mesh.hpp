// Oracle (test infrastructure only): cubical-cell mesh with one optional level
// of static refinement, and its neighbour table found by geometric search.
//
// Written from the paper's description of the tree (Sec. 4): leaf cells and
// nodes, six neighbour indices per cell, the index of the same-level node
// stored in place of a split neighbour, and a level jump of at most one.
//
// Conventions shared with the library only as an interface format:
//  * cells are listed by base cell in lexicographic order (x fastest); an
//    unrefined base cell is one cell, a refined base cell is replaced by its
//    2^d children in the order A..H of Sec. 4.2 / Appendix F (child bit of
//    axis a is bit a of the child number, so x is fastest);
//  * neighbour table entry [side][cell], side = 2*axis + (0 for -, 1 for +):
//    >= 0 a leaf cell, -1 no neighbour (non-periodic boundary),
//    <= -2 the node -(entry+2) (the neighbour at the same level is split).
#pragma once
#include <array>
#include <cmath>
#include <cstdint>
#include <map>
#include <stdexcept>
#include <vector>

namespace orc {

enum { BC_PERIODIC = 0, BC_TRANSMISSIVE = 1 };

struct Mesh {
  int dim = 2;
  int n[3] = {1, 1, 1};
  double lo[3] = {0, 0, 0}, hi[3] = {1, 1, 1};
  int bc[3] = {BC_PERIODIC, BC_PERIODIC, BC_PERIODIC};
  double dx0 = 1.0;  // base edge length

  int ncells = 0, nnodes = 0;
  std::vector<int> level;                        // per cell
  std::vector<std::array<int, 3>> coord;         // integer position at the cell's level
  std::vector<std::array<int, 3>> node_coord;    // integer position of a node (level 0)
  std::vector<std::vector<int>> node_children;   // 2^d child cell ids per node
  std::vector<int32_t> nbr;                      // [2*dim][ncells]

  int nsides() const { return 2 * dim; }
  double dx(int c) const { return dx0 / (double)(1 << level[c]); }
  double center(int c, int a) const { return lo[a] + (coord[c][a] + 0.5) * dx(c); }

  void build(int dim_, const int* n_, const double* lo_, const double* hi_, const int* bc_,
             int n_boxes, const int* boxes) {
    dim = dim_;
    for (int a = 0; a < 3; ++a) {
      n[a] = a < dim ? n_[a] : 1;
      lo[a] = a < dim ? lo_[a] : 0.0;
      hi[a] = a < dim ? hi_[a] : 1.0;
      bc[a] = a < dim ? bc_[a] : BC_PERIODIC;
    }
    dx0 = (hi[0] - lo[0]) / n[0];
    for (int a = 1; a < dim; ++a) {
      double d = (hi[a] - lo[a]) / n[a];
      if (std::fabs(d - dx0) > 1e-12 * dx0) throw std::runtime_error("cells must be cubical");
    }
    auto refined = [&](int ix, int iy, int iz) {
      for (int b = 0; b < n_boxes; ++b) {
        const int* bx = boxes + 2 * dim * b;  // lo[0..dim), hi[0..dim) inclusive
        int p[3] = {ix, iy, iz};
        bool in = true;
        for (int a = 0; a < dim; ++a) in = in && p[a] >= bx[a] && p[a] <= bx[dim + a];
        if (in) return true;
      }
      return false;
    };
    const int nch = 1 << dim;
    for (int iz = 0; iz < n[2]; ++iz)
      for (int iy = 0; iy < n[1]; ++iy)
        for (int ix = 0; ix < n[0]; ++ix) {
          if (!refined(ix, iy, iz)) {
            level.push_back(0);
            coord.push_back({ix, iy, iz});
          } else {
            std::vector<int> kids;
            for (int s = 0; s < nch; ++s) {
              level.push_back(1);
              coord.push_back({2 * ix + (s & 1), 2 * iy + ((s >> 1) & 1),
                               dim == 3 ? 2 * iz + ((s >> 2) & 1) : 0});
              kids.push_back((int)level.size() - 1);
            }
            node_coord.push_back({ix, iy, iz});
            node_children.push_back(kids);
          }
        }
    ncells = (int)level.size();
    nnodes = (int)node_coord.size();
    find_neighbours();
  }

  // Geometric search: the same-size region next to each face is looked up
  // among the leaf cells of its level, then among coarser leaves containing
  // it, then among the nodes.
  void find_neighbours() {
    std::map<std::array<int, 4>, int> leaf, node;
    for (int c = 0; c < ncells; ++c)
      leaf[{level[c], coord[c][0], coord[c][1], coord[c][2]}] = c;
    for (int m = 0; m < nnodes; ++m)
      node[{0, node_coord[m][0], node_coord[m][1], node_coord[m][2]}] = m;
    nbr.assign((size_t)nsides() * ncells, -1);
    for (int c = 0; c < ncells; ++c) {
      const int l = level[c];
      for (int a = 0; a < dim; ++a)
        for (int s = 0; s < 2; ++s) {
          std::array<int, 3> p = coord[c];
          p[a] += s ? 1 : -1;
          const int extent = n[a] << l;
          bool outside = false;
          if (p[a] < 0 || p[a] >= extent) {
            if (bc[a] == BC_PERIODIC)
              p[a] = (p[a] + extent) % extent;
            else
              outside = true;
          }
          int32_t v = -1;
          if (!outside) {
            auto it = leaf.find({l, p[0], p[1], p[2]});
            if (it != leaf.end()) {
              v = it->second;
            } else if (l > 0 && leaf.count({l - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1})) {
              v = leaf[{l - 1, p[0] >> 1, p[1] >> 1, p[2] >> 1}];
            } else {
              auto jt = node.find({l, p[0], p[1], p[2]});
              if (jt == node.end()) throw std::runtime_error("level jump larger than one");
              v = -(jt->second + 2);
            }
          }
          nbr[(size_t)(2 * a + s) * ncells + c] = v;
        }
    }
  }
};

}  // namespace orc
