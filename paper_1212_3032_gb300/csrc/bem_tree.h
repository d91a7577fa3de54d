// Cluster tree and block tree of the hierarchical (block low-rank) operator.
//
// The paper accelerates the matrix-vector product with pFFT and names the
// H-matrix method as the alternative (Sec. 4.1). This library uses the
// H-matrix form: elements are ordered by a geometric bisection tree; a pair
// of clusters (tau, sigma) is admissible (low rank) when
//   min(diam tau, diam sigma) <= eta_adm * dist(tau, sigma)
// and no element pair in it falls in the near-singular quadrature band; the
// remaining leaf pairs are dense near-field blocks.
#pragma once

#include <cstdint>
#include <vector>

namespace bem {

struct Cluster {
  int begin = 0, end = 0;  // element range in tree order
  double bmin[3] = {0, 0, 0}, bmax[3] = {0, 0, 0};
  double hmax = 0;         // largest element size h inside
  int child[2] = {-1, -1};
  bool leaf() const { return child[0] < 0; }
  int size() const { return end - begin; }
};

struct BlockPair {
  int tau, sigma;  // cluster indices (rows, columns)
};

struct ClusterTree {
  std::vector<int> perm;      // tree position -> caller element index
  std::vector<int> iperm;     // caller element index -> tree position
  std::vector<Cluster> nodes; // nodes[0] is the root
  std::vector<int> leaf_of;   // tree position -> leaf node index
  std::vector<BlockPair> near, far;
};

// centroid: ne x 3, h: ne (caller order). rho2_near: squared near-singular
// band threshold (pairs closer than this never enter an admissible block).
void build_cluster_tree(const double* centroid, const double* h, int ne, int leaf_size,
                        double eta_adm, double rho2_near, bool all_dense, ClusterTree& out);

}  // namespace bem
