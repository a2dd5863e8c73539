// Closed forms of the cluster-tree order (Sec. 3.2.2 index sets; the KD / Morton order of
// Sec. 5.2), for the device kernels of tree.cu and the host-only planning query.
//
//   * 1-D: the interior nodes in natural order.
//   * 2-D: Morton (Z) order, x-index bit b at key bit 2b and y-index bit b at key bit 2b+1; the
//     spatial position of a point is the rank of its key among the G^2 keys of the grid, which
//     morton_rank counts bit by bit without a sort (on a 2^q x 2^q grid it is the key itself).
//   * every node [lo, hi) of spatial positions splits at lo + (hi - lo) / 2, tau times; a leaf
//     of nvar variables holds [variable 1 of its points, variable 2 of the same points].
#pragma once

namespace hodlr {

struct TreeDesc {
  int dim, G, nvar, Ns, tau;
  int slot;   // rows of a leaf slot of the tree layout (nvar x the largest leaf)
};

__host__ __device__ inline int tree_nbits(int G) {
  int n = 1;
  while ((1 << n) < G) ++n;
  return n;
}

// |[lo, lo + w) intersected with [0, G)| for lo >= 0
__host__ __device__ inline long long tree_span(long long lo, long long w, long long G) {
  if (lo >= G) return 0;
  return (lo + w < G ? lo + w : G) - lo;
}

// Number of points (x, y) of the G x G grid whose Morton key is below the key of (ix, iy).
// Walking the key from its top bit down, every 1 bit of the key adds the points that agree with
// (ix, iy) on all higher key bits and have a 0 here: their x (y) values fill an aligned block of
// 2^(free low bits) consecutive indices, cut at G.
__host__ __device__ inline long long morton_rank(int ix, int iy, int G, int nbits) {
  long long r = 0;
  int fx = nbits, fy = nbits;   // low bits of x (y) not yet fixed by the walk
  for (int j = 2 * nbits - 1; j >= 0; --j) {
    const int b = j >> 1;
    if (j & 1) {   // bit b of y
      if ((iy >> b) & 1) {
        const long long y0 = (long long)(iy >> (b + 1)) << (b + 1);
        const long long x0 = (long long)(ix >> fx) << fx;
        r += tree_span(y0, 1LL << b, G) * tree_span(x0, 1LL << fx, G);
      }
      fy = b;
    } else {       // bit b of x
      if ((ix >> b) & 1) {
        const long long x0 = (long long)(ix >> (b + 1)) << (b + 1);
        const long long y0 = (long long)(iy >> fy) << fy;
        r += tree_span(x0, 1LL << b, G) * tree_span(y0, 1LL << fy, G);
      }
      fx = b;
    }
  }
  return r;
}

// spatial position of the natural spatial index p
__host__ __device__ inline int tree_spatial_pos(const TreeDesc& t, int p) {
  if (t.dim == 1) return p;
  return (int)morton_rank(p % t.G, p / t.G, t.G, tree_nbits(t.G));
}

// leaf holding spatial position s, and its range [lo, hi) of spatial positions
__host__ __device__ inline int tree_leaf(const TreeDesc& t, int s, int& lo, int& hi) {
  lo = 0;
  hi = t.Ns;
  int b = 0;
  for (int d = 0; d < t.tau; ++d) {
    const int mid = lo + (hi - lo) / 2;
    if (s < mid) { hi = mid; b = 2 * b; }
    else { lo = mid; b = 2 * b + 1; }
  }
  return b;
}

}  // namespace hodlr
