// Hilbert-curve re-sort of the cell arrays (Sussman, arXiv 1702.02939,
// Sec. 2.B): cells that are close in space are placed close in memory, so the
// gathers of neighbour positions, rings and force sets stay local.  Each cell
// gets the position along a Hilbert curve of its replica's sort grid; a
// counting sort by that key gives the permutation, and one kernel moves every
// per-cell array and renames the ring entries.  Results do not depend on the
// storage order: rings are kept in canonical form by cell tag.
#include "cg_device.cuh"
#include "cg_kernels.h"

namespace cgk {

__global__ void k_sort_keys(SortArgs g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int cur = g.ctl->cur;
  const Rep R = g.reps[g.rep[i]];
  const unsigned side = 1u << R.hord;
  unsigned gx = (unsigned)(g.X[(size_t)cur * g.n + i] >> R.hshift);
  unsigned gy = (unsigned)(g.Y[(size_t)cur * g.n + i] >> R.hshift);
  gx = gx >= side ? side - 1 : gx;
  gy = gy >= side ? side - 1 : gy;
  const int key = R.hkey0 + (int)hilbert_index(R.hord, gx, gy);
  g.key[i] = key;
  g.rank[i] = atomicAdd(&g.key_count[key], 1);
}

__global__ void k_sort_perm(SortArgs g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const int k = g.key[i];
  g.perm[i] = bin_begin(g.key_start, g.key_partials, k) + g.rank[i];
  g.key_count[k] = 0;
}

__global__ void k_sort_move(SortArgs g) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= g.n) return;
  const size_t N = (size_t)g.n;
  const int cur = g.ctl->cur, alt = cur ^ 1;
  const int j = g.perm[i];
  g.x[alt * N + j] = g.x[cur * N + i];
  g.y[alt * N + j] = g.y[cur * N + i];
  g.X[alt * N + j] = g.X[cur * N + i];
  g.Y[alt * N + j] = g.Y[cur * N + i];
  g.theta_alt[j] = g.theta[i];
  g.p0_alt[j] = g.p0[i];
  g.v0_alt[j] = g.v0[i];
  g.tag_alt[j] = g.tag[i];
  g.nid_alt[j] = g.nid[i];
  g.rep_alt[j] = g.rep[i];
  const int m = g.cnt[i];
  g.cnt_alt[j] = m;
  for (int a = 0; a < CG_RING; ++a) {
    const int v = g.nbr[(size_t)i * CG_RING + a];
    g.nbr_alt[(size_t)j * CG_RING + a] = (a < m && v >= 0 && v < g.n) ? g.perm[v] : -1;
  }
}

__global__ void k_sort_flip(Ctl* ctl) { ctl->cur ^= 1; }

void launch_sort(const SortArgs& a, cudaStream_t st) {
  if (a.n <= 0) return;
  const int blocks = (a.n + 255) / 256;
  k_sort_keys<<<blocks, 256, 0, st>>>(a);
  CellListArgs sc{};
  sc.n = a.n;
  sc.nbins = a.nkeys;
  sc.ctl = a.ctl;
  sc.bin_count = a.key_count;
  sc.bin_start = a.key_start;
  sc.scan_partials = a.key_partials;
  sc.only_if_flagged = 0;
  launch_scan(sc, st);
  k_sort_perm<<<blocks, 256, 0, st>>>(a);
  k_sort_move<<<blocks, 256, 0, st>>>(a);
  k_sort_flip<<<1, 1, 0, st>>>(a.ctl);
  const size_t N = (size_t)a.n;
  cudaMemcpyAsync(a.theta, a.theta_alt, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.p0, a.p0_alt, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.v0, a.v0_alt, N * sizeof(double), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.tag, a.tag_alt, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.nid, a.nid_alt, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.rep, a.rep_alt, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.cnt, a.cnt_alt, N * sizeof(int), cudaMemcpyDeviceToDevice, st);
  cudaMemcpyAsync(a.nbr, a.nbr_alt, N * CG_RING * sizeof(int), cudaMemcpyDeviceToDevice, st);
}

}  // namespace cgk
