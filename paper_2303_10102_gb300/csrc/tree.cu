// Cluster-tree order and layout maps on the device (Sec. 3.2.2 index sets; the KD / Morton
// order of Sec. 5.2).  One thread per grid point finds its spatial position by the closed-form
// Morton rank and its leaf by the halving walk (tree.cuh), and writes the maps of the padded
// tree layout; no sort and no host pass over the points.
#include "common.cuh"
#include "ops.h"

namespace hodlr {
namespace {

__global__ void tree_order_kernel(TreeDesc t, int* permpad, int* rowid, int* real2pad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= t.Ns) return;
  const int s = tree_spatial_pos(t, p);
  int lo, hi;
  const int b = tree_leaf(t, s, lo, hi);
  for (int v = 0; v < t.nvar; ++v) {
    const int k = v * (hi - lo) + (s - lo);   // row within the leaf
    const int pos = t.nvar * lo + k;          // real tree position
    const int slot = b * t.slot + k;          // row of the padded tree layout
    permpad[slot] = v * t.Ns + p;
    if (rowid) rowid[slot] = pos;
    real2pad[pos] = slot;
  }
}

// natural index -> row of a physics panel whose variable blocks are Ns x qc
__global__ void tree_phys_perm_kernel(const int* permpad, int N, int Ns, int nvar, int qc, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int n = permpad[i];
  out[i] = n < 0 ? -1 : (nvar == 1 ? n : (int)((long long)(n % Ns) + (long long)(n / Ns) * Ns * qc));
}

__global__ void tree_level_mask_kernel(int N, int msize, const int* rowid, unsigned char* mask) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  mask[i] = ((i / msize) & 1) && (!rowid || rowid[i] >= 0) ? 1 : 0;
}

}  // namespace

void tree_order(const TreeDesc& t, int N, int* permpad, int* rowid, int* real2pad, cudaStream_t st) {
  HODLR_CUDA(cudaMemsetAsync(permpad, 0xff, sizeof(int) * (size_t)N, st));   // -1: padding rows
  if (rowid) HODLR_CUDA(cudaMemsetAsync(rowid, 0xff, sizeof(int) * (size_t)N, st));
  tree_order_kernel<<<cdiv(t.Ns, 256), 256, 0, st>>>(t, permpad, rowid, real2pad);
  check_launch("tree_order");
}

void tree_phys_perm(const int* permpad, int N, int Ns, int nvar, int qc, int* out, cudaStream_t st) {
  tree_phys_perm_kernel<<<cdiv(N, 256), 256, 0, st>>>(permpad, N, Ns, nvar, qc, out);
  check_launch("tree_phys_perm");
}

void tree_level_mask(int N, int msize, const int* rowid, unsigned char* mask, cudaStream_t st) {
  tree_level_mask_kernel<<<cdiv(N, 256), 256, 0, st>>>(N, msize, rowid, mask);
  check_launch("tree_level_mask");
}

}  // namespace hodlr
