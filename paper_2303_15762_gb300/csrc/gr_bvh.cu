// Linear BVH construction on the GPU (Karras, "Maximizing Parallelism in the
// Construction of BVHs, Octrees, and k-d Trees", HPG 2012).
//
// Propagation of a generalized ray under the interactive simplification of the
// paper (Sec. 7.2) is ray tracing, which needs a spatial subdivision of the
// scene (Sec. 1 motivates locality by exactly this).  The paper does not
// describe its structure; this build uses a binary LBVH:
//   centroid bounds -> 30-bit Morton codes -> 64-bit keys (morton << 32 | id)
//   -> bitonic sort -> Karras hierarchy -> bottom-up child boxes.
// Every step is integer work or exact FP32 (min/max, and centroid/quantisation
// arithmetic in explicitly rounded single precision), so the result is
// deterministic and reproducible bit for bit by a CPU build of the same
// algorithm.
#include "gr_build.h"

namespace gr {

namespace {

__device__ __forceinline__ unsigned expand_bits(unsigned v) {
  v = (v * 0x00010001u) & 0xFF0000FFu;
  v = (v * 0x00000101u) & 0x0F00F00Fu;
  v = (v * 0x00000011u) & 0xC30C30C3u;
  v = (v * 0x00000005u) & 0x49249249u;
  return v;
}

__global__ void k_centroids(const float* __restrict__ verts, int n, float4* __restrict__ cen) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float* v = verts + 9 * i;
  float cx = __fdiv_rn(__fadd_rn(__fadd_rn(v[0], v[3]), v[6]), 3.0f);
  float cy = __fdiv_rn(__fadd_rn(__fadd_rn(v[1], v[4]), v[7]), 3.0f);
  float cz = __fdiv_rn(__fadd_rn(__fadd_rn(v[2], v[5]), v[8]), 3.0f);
  cen[i] = make_float4(cx, cy, cz, 0.0f);
}

// One block reduces the centroid bounds (exact min/max).
__global__ void k_bounds(const float4* __restrict__ cen, int n, float* __restrict__ out6) {
  __shared__ float s[6][1024];
  float lo[3] = {3.4e38f, 3.4e38f, 3.4e38f}, hi[3] = {-3.4e38f, -3.4e38f, -3.4e38f};
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    float4 c = cen[i];
    lo[0] = fminf(lo[0], c.x);
    lo[1] = fminf(lo[1], c.y);
    lo[2] = fminf(lo[2], c.z);
    hi[0] = fmaxf(hi[0], c.x);
    hi[1] = fmaxf(hi[1], c.y);
    hi[2] = fmaxf(hi[2], c.z);
  }
  for (int a = 0; a < 3; ++a) {
    s[a][threadIdx.x] = lo[a];
    s[3 + a][threadIdx.x] = hi[a];
  }
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) {
      for (int a = 0; a < 3; ++a) {
        s[a][threadIdx.x] = fminf(s[a][threadIdx.x], s[a][threadIdx.x + w]);
        s[3 + a][threadIdx.x] = fmaxf(s[3 + a][threadIdx.x], s[3 + a][threadIdx.x + w]);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) out6[threadIdx.x] = s[threadIdx.x][0];
}

__global__ void k_morton(const float4* __restrict__ cen, int n, int n_pad, const float* __restrict__ b6,
                         unsigned long long* __restrict__ keys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_pad) return;
  if (i >= n) {
    keys[i] = ~0ull;
    return;
  }
  float4 c = cen[i];
  float cc[3] = {c.x, c.y, c.z};
  unsigned q[3];
  for (int a = 0; a < 3; ++a) {
    float ext = __fsub_rn(b6[3 + a], b6[a]);
    float t = ext > 0.0f ? __fdiv_rn(__fsub_rn(cc[a], b6[a]), ext) : 0.0f;
    int qi = (int)__fmul_rn(t, 1024.0f);
    qi = qi < 0 ? 0 : (qi > 1023 ? 1023 : qi);
    q[a] = (unsigned)qi;
  }
  unsigned m = expand_bits(q[0]) * 4u + expand_bits(q[1]) * 2u + expand_bits(q[2]);
  keys[i] = ((unsigned long long)m << 32) | (unsigned)i;
}

// Bitonic sorting network (ascending): stages with j >= 1024 run one global
// pass each; all stages with j < 1024 of one k run in shared memory.
__global__ void k_bitonic_global(unsigned long long* keys, int n_pad, int j, int k) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_pad / 2) return;
  int a = 2 * j * (t / j) + (t % j);
  int b = a + j;
  unsigned long long x = keys[a], y = keys[b];
  bool up = (a & k) == 0;
  if ((x > y) == up) {
    keys[a] = y;
    keys[b] = x;
  }
}

__global__ void k_bitonic_shared(unsigned long long* keys, int n_pad, int k_first, int k_last) {
  __shared__ unsigned long long s[2048];
  int base = blockIdx.x * 2048;
  s[threadIdx.x] = keys[base + threadIdx.x];
  s[threadIdx.x + 1024] = keys[base + threadIdx.x + 1024];
  __syncthreads();
  for (int k = k_first; k <= k_last; k <<= 1) {
    int jstart = k >> 1;
    if (jstart > 1024) jstart = 1024;
    for (int j = jstart; j >= 1; j >>= 1) {
      int t = threadIdx.x;
      int a = 2 * j * (t / j) + (t % j);
      int b = a + j;
      unsigned long long x = s[a], y = s[b];
      bool up = ((base + a) & k) == 0;
      if ((x > y) == up) {
        s[a] = y;
        s[b] = x;
      }
      __syncthreads();
    }
  }
  keys[base + threadIdx.x] = s[threadIdx.x];
  keys[base + threadIdx.x + 1024] = s[threadIdx.x + 1024];
}

__device__ __forceinline__ int delta(const unsigned long long* keys, int n, int i, int j) {
  if (j < 0 || j > n - 1) return -1;
  return __clzll(keys[i] ^ keys[j]);
}

// Internal node i of the Karras hierarchy: its key range, split and children.
__global__ void k_hierarchy(const unsigned long long* __restrict__ keys, int n, float* __restrict__ nodes,
                            int* __restrict__ leaf_parent, int* __restrict__ node_parent) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  int d = (delta(keys, n, i, i + 1) - delta(keys, n, i, i - 1)) >= 0 ? 1 : -1;
  int dmin = delta(keys, n, i, i - d);
  int lmax = 2;
  while (delta(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
  int l = 0;
  for (int t = lmax / 2; t >= 1; t /= 2)
    if (delta(keys, n, i, i + (l + t) * d) > dmin) l += t;
  int j = i + l * d;
  int dnode = delta(keys, n, i, j);
  int s = 0, t = l;
  do {
    t = (t + 1) >> 1;
    if (delta(keys, n, i, i + (s + t) * d) > dnode) s += t;
  } while (t > 1);
  int gamma = i + s * d + (d < 0 ? -1 : 0);
  int lo = i < j ? i : j, hi = i < j ? j : i;
  int lref = (lo == gamma) ? (gamma | 0x80000000) : gamma;
  int rref = (hi == gamma + 1) ? ((gamma + 1) | 0x80000000) : (gamma + 1);
  float* N = nodes + 16 * i;
  N[12] = __int_as_float(lref);
  N[13] = __int_as_float(rref);
  N[15] = 0.0f;
  if (lref < 0)
    leaf_parent[gamma] = i;
  else
    node_parent[gamma] = i;
  if (rref < 0)
    leaf_parent[gamma + 1] = i;
  else
    node_parent[gamma + 1] = i;
  if (i == 0) N[14] = __int_as_float(-1);
}

// Gather the triangles into leaf order; tri[3i].w carries the original id.
__global__ void k_reorder(const unsigned long long* __restrict__ keys, int n, const float* __restrict__ verts,
                          const int* __restrict__ tri_mat, float4* __restrict__ tri, int* __restrict__ tmat) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int id = (int)(keys[i] & 0xffffffffu);
  const float* v = verts + 9 * id;
  tri[3 * i] = make_float4(v[0], v[1], v[2], __int_as_float(id));
  tri[3 * i + 1] = make_float4(v[3], v[4], v[5], 0.0f);
  tri[3 * i + 2] = make_float4(v[6], v[7], v[8], 0.0f);
  tmat[i] = tri_mat[id];
}

__device__ __forceinline__ void write_box(float* nodes, int node, int side, const float lo[3], const float hi[3]) {
  float* N = nodes + 16 * node + 6 * side;
  __stcg(N + 0, lo[0]);
  __stcg(N + 1, lo[1]);
  __stcg(N + 2, lo[2]);
  __stcg(N + 3, hi[0]);
  __stcg(N + 4, hi[1]);
  __stcg(N + 5, hi[2]);
}

// Bottom-up child boxes: each leaf walks to the root; the second thread to
// reach a node merges its two child boxes (exact FP32 min/max, so the result
// does not depend on the arrival order).
__global__ void k_boxes(const float4* __restrict__ tri, int n, float* nodes, const int* __restrict__ leaf_parent,
                        const int* __restrict__ node_parent, int* flags) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float4 a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
  float lo[3] = {fminf(fminf(a.x, b.x), c.x), fminf(fminf(a.y, b.y), c.y), fminf(fminf(a.z, b.z), c.z)};
  float hi[3] = {fmaxf(fmaxf(a.x, b.x), c.x), fmaxf(fmaxf(a.y, b.y), c.y), fmaxf(fmaxf(a.z, b.z), c.z)};
  int child = i | 0x80000000;
  int p = leaf_parent[i];
  int guard = n;  // at most n-1 ancestors
  while (p >= 0 && --guard >= 0) {
    int lref = __float_as_int(__ldcg(nodes + 16 * p + 12));
    int side = (lref == child) ? 0 : 1;
    write_box(nodes, p, side, lo, hi);
    __threadfence();
    int old = atomicAdd(flags + p, 1);
    if (old == 0) return;  // the sibling subtree is not finished yet
    __threadfence();
    const float* N = nodes + 16 * p;
    for (int k = 0; k < 3; ++k) {
      lo[k] = fminf(__ldcg(N + k), __ldcg(N + 6 + k));
      hi[k] = fmaxf(__ldcg(N + 3 + k), __ldcg(N + 9 + k));
    }
    child = p;
    p = (p == 0) ? -1 : node_parent[p];
  }
}

inline cudaError_t launch_sort(unsigned long long* keys, int n_pad, cudaStream_t st) {
  // n_pad is a power of two >= 2048
  int blocks_sh = n_pad / 2048;
  k_bitonic_shared<<<blocks_sh, 1024, 0, st>>>(keys, n_pad, 2, 2048);
  for (int k = 4096; k <= n_pad; k <<= 1) {
    for (int j = k >> 1; j >= 2048; j >>= 1) {
      int threads = n_pad / 2;
      k_bitonic_global<<<(threads + 255) / 256, 256, 0, st>>>(keys, n_pad, j, k);
    }
    k_bitonic_shared<<<blocks_sh, 1024, 0, st>>>(keys, n_pad, k, k);
  }
  return cudaGetLastError();
}

}  // namespace

// Build the BVH of `n` triangles (device arrays verts [n][9], tri_mat [n]).
// Outputs (device, caller-allocated): tri [n][3] float4, tmat [n], nodes
// [(n-1)][16] floats, keys [n_pad].  Scratch is allocated here and freed
// before return (stream-ordered).
cudaError_t build_lbvh(const float* verts, const int* tri_mat, int n, float4* tri, int* tmat, float* nodes,
                       unsigned long long* keys_out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int n_pad = 2048;
  while (n_pad < n) n_pad <<= 1;
  float4* cen = nullptr;
  float* b6 = nullptr;
  unsigned long long* keys = nullptr;
  int *leaf_parent = nullptr, *node_parent = nullptr, *flags = nullptr;
  cudaError_t e = cudaSuccess;
#define GR_TRY(x)                 \
  do {                            \
    e = (x);                      \
    if (e != cudaSuccess) goto done; \
  } while (0)
  GR_TRY(cudaMallocAsync(&cen, sizeof(float4) * n, st));
  GR_TRY(cudaMallocAsync(&b6, sizeof(float) * 6, st));
  GR_TRY(cudaMallocAsync(&keys, sizeof(unsigned long long) * n_pad, st));
  GR_TRY(cudaMallocAsync(&leaf_parent, sizeof(int) * n, st));
  GR_TRY(cudaMallocAsync(&node_parent, sizeof(int) * n, st));
  GR_TRY(cudaMallocAsync(&flags, sizeof(int) * n, st));
  GR_TRY(cudaMemsetAsync(flags, 0, sizeof(int) * n, st));
  GR_TRY(cudaMemsetAsync(leaf_parent, 0xff, sizeof(int) * n, st));
  GR_TRY(cudaMemsetAsync(node_parent, 0xff, sizeof(int) * n, st));
  k_centroids<<<(n + 255) / 256, 256, 0, st>>>(verts, n, cen);
  k_bounds<<<1, 1024, 0, st>>>(cen, n, b6);
  k_morton<<<(n_pad + 255) / 256, 256, 0, st>>>(cen, n, n_pad, b6, keys);
  GR_TRY(cudaGetLastError());
  GR_TRY(launch_sort(keys, n_pad, st));
  if (n > 1) {
    GR_TRY(cudaMemsetAsync(nodes, 0, sizeof(float) * 16 * (size_t)(n - 1), st));
    k_hierarchy<<<(n - 1 + 255) / 256, 256, 0, st>>>(keys, n, nodes, leaf_parent, node_parent);
  }
  k_reorder<<<(n + 255) / 256, 256, 0, st>>>(keys, n, verts, tri_mat, tri, tmat);
  if (n > 1) k_boxes<<<(n + 255) / 256, 256, 0, st>>>(tri, n, nodes, leaf_parent, node_parent, flags);
  GR_TRY(cudaGetLastError());
  if (keys_out) GR_TRY(cudaMemcpyAsync(keys_out, keys, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st));
done:
  if (cen) cudaFreeAsync(cen, st);
  if (b6) cudaFreeAsync(b6, st);
  if (keys) cudaFreeAsync(keys, st);
  if (leaf_parent) cudaFreeAsync(leaf_parent, st);
  if (node_parent) cudaFreeAsync(node_parent, st);
  if (flags) cudaFreeAsync(flags, st);
#undef GR_TRY
  return e;
}

}  // namespace gr
