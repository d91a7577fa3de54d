// Host construction of the cluster tree (median bisection along the longest
// bounding-box axis) and of the block tree (near / admissible far pairs).
#include "bem_tree.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <numeric>

namespace bem {

static std::atomic<long long> g_launches{0};
bool count_if(bool c) {
  if (c) g_launches.fetch_add(1, std::memory_order_relaxed);
  return c;
}
long long launch_count() { return g_launches.load(std::memory_order_relaxed); }

namespace {

struct Builder {
  const double* c;
  const double* h;
  int leaf;
  std::vector<int> idx;
  std::vector<Cluster> nodes;

  void bbox(Cluster& cl) {
    for (int a = 0; a < 3; ++a) {
      cl.bmin[a] = INFINITY;
      cl.bmax[a] = -INFINITY;
    }
    cl.hmax = 0;
    for (int k = cl.begin; k < cl.end; ++k) {
      int e = idx[k];
      for (int a = 0; a < 3; ++a) {
        cl.bmin[a] = std::min(cl.bmin[a], c[3 * e + a]);
        cl.bmax[a] = std::max(cl.bmax[a], c[3 * e + a]);
      }
      cl.hmax = std::max(cl.hmax, h[e]);
    }
  }

  int build(int begin, int end) {
    int id = (int)nodes.size();
    nodes.emplace_back();
    nodes[id].begin = begin;
    nodes[id].end = end;
    bbox(nodes[id]);
    if (end - begin > leaf) {
      int axis = 0;
      double ext = -1;
      for (int a = 0; a < 3; ++a) {
        double e = nodes[id].bmax[a] - nodes[id].bmin[a];
        if (e > ext) {
          ext = e;
          axis = a;
        }
      }
      int mid = begin + (end - begin) / 2;
      // deterministic median split: order by (coordinate, element index)
      std::nth_element(idx.begin() + begin, idx.begin() + mid, idx.begin() + end,
                       [&](int p, int q) {
                         double cp = c[3 * p + axis], cq = c[3 * q + axis];
                         return cp < cq || (cp == cq && p < q);
                       });
      int l = build(begin, mid);
      int r = build(mid, end);
      nodes[id].child[0] = l;
      nodes[id].child[1] = r;
    }
    return id;
  }
};

double diam(const Cluster& a) {
  double s = 0;
  for (int k = 0; k < 3; ++k) s += (a.bmax[k] - a.bmin[k]) * (a.bmax[k] - a.bmin[k]);
  return std::sqrt(s);
}

double dist2(const Cluster& a, const Cluster& b) {
  double s = 0;
  for (int k = 0; k < 3; ++k) {
    double d = std::max(0.0, std::max(a.bmin[k] - b.bmax[k], b.bmin[k] - a.bmax[k]));
    s += d * d;
  }
  return s;
}

}  // namespace

void build_cluster_tree(const double* centroid, const double* h, int ne, int leaf_size,
                        double eta_adm, double rho2_near, bool all_dense, ClusterTree& out) {
  Builder b;
  b.c = centroid;
  b.h = h;
  b.leaf = std::max(1, leaf_size);
  b.idx.resize(ne);
  std::iota(b.idx.begin(), b.idx.end(), 0);
  b.build(0, ne);
  out.nodes = std::move(b.nodes);
  out.perm = std::move(b.idx);
  out.iperm.assign(ne, 0);
  for (int k = 0; k < ne; ++k) out.iperm[out.perm[k]] = k;
  out.leaf_of.assign(ne, -1);
  for (int id = 0; id < (int)out.nodes.size(); ++id) {
    const Cluster& cl = out.nodes[id];
    if (cl.leaf())
      for (int k = cl.begin; k < cl.end; ++k) out.leaf_of[k] = id;
  }
  out.near.clear();
  out.far.clear();
  const auto& nodes = out.nodes;
  // explicit stack instead of recursion (deep trees on large meshes)
  std::vector<BlockPair> stack{{0, 0}};
  while (!stack.empty()) {
    BlockPair p = stack.back();
    stack.pop_back();
    const Cluster& t = nodes[p.tau];
    const Cluster& s = nodes[p.sigma];
    double d2 = dist2(t, s);
    double hm = std::max(t.hmax, s.hmax);
    bool adm = !all_dense && d2 > 0 &&
               std::min(diam(t), diam(s)) <= eta_adm * std::sqrt(d2) &&
               d2 > rho2_near * hm * hm * 1.0001;
    if (adm) {
      out.far.push_back(p);
    } else if (t.leaf() && s.leaf()) {
      out.near.push_back(p);
    } else if (t.leaf()) {
      stack.push_back({p.tau, s.child[1]});
      stack.push_back({p.tau, s.child[0]});
    } else if (s.leaf()) {
      stack.push_back({t.child[1], p.sigma});
      stack.push_back({t.child[0], p.sigma});
    } else {
      stack.push_back({t.child[1], s.child[1]});
      stack.push_back({t.child[1], s.child[0]});
      stack.push_back({t.child[0], s.child[1]});
      stack.push_back({t.child[0], s.child[0]});
    }
  }
  // deterministic order: near blocks by (row leaf begin, col begin)
  auto key = [&](const BlockPair& a, const BlockPair& b2) {
    const Cluster &ta = nodes[a.tau], &sa = nodes[a.sigma];
    const Cluster &tb = nodes[b2.tau], &sb = nodes[b2.sigma];
    if (ta.begin != tb.begin) return ta.begin < tb.begin;
    if (sa.begin != sb.begin) return sa.begin < sb.begin;
    return ta.end < tb.end;
  };
  std::sort(out.near.begin(), out.near.end(), key);
  std::sort(out.far.begin(), out.far.end(), key);
}

}  // namespace bem
