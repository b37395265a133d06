// BVH construction on the GPU.
//
// Propagation of a generalized ray under the interactive simplification of the
// paper (Sec. 7.2) is ray tracing, which needs a spatial subdivision of the
// scene (Sec. 1 motivates locality by exactly this).  The paper does not
// describe its structure; the tree here is built by
//   centroid bounds -> 30-bit Morton codes -> 64-bit keys (morton << 32 | id)
//   -> bitonic sort -> agglomerative clustering along the Morton order
//   (PLOC: Meister & Bittner, "Parallel Locally-Ordered Clustering for
//   Bounding Volume Hierarchy Construction", IEEE TVCG 2018): each cluster
//   picks the neighbour within a window of +-8 whose merged box has the least
//   surface area; mutual nearest neighbours merge, the array is compacted, and
//   the loop repeats until one cluster remains.
// Every step is integer work or exact FP32 (min/max, and centroid,
// quantisation and surface-area arithmetic in explicitly rounded single
// precision), ties go to the lower index and node indices come from prefix
// sums, so the result is deterministic and reproducible bit for bit by a CPU
// build of the same algorithm.
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

// ---- PLOC
constexpr int kPlocRadius = 8;

struct Box6 {
  float lo[3], hi[3];
};

__device__ __forceinline__ Box6 box_union(const Box6& a, const Box6& b) {
  Box6 r;
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = fminf(a.lo[k], b.lo[k]);
    r.hi[k] = fmaxf(a.hi[k], b.hi[k]);
  }
  return r;
}

// Half surface area, rounded step by step: ((dx dy) + (dy dz)) + (dz dx).
__device__ __forceinline__ float half_area_rn(const Box6& b) {
  const float dx = __fsub_rn(b.hi[0], b.lo[0]), dy = __fsub_rn(b.hi[1], b.lo[1]), dz = __fsub_rn(b.hi[2], b.lo[2]);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dy), __fmul_rn(dy, dz)), __fmul_rn(dz, dx));
}

__device__ __forceinline__ Box6 load_box(const float* B, int i) {
  Box6 r;
  for (int k = 0; k < 3; ++k) {
    r.lo[k] = B[6 * i + k];
    r.hi[k] = B[6 * i + 3 + k];
  }
  return r;
}
__device__ __forceinline__ void store_box(float* B, int i, const Box6& b) {
  for (int k = 0; k < 3; ++k) {
    B[6 * i + k] = b.lo[k];
    B[6 * i + 3 + k] = b.hi[k];
  }
}

__global__ void k_leaf_clusters(const float4* __restrict__ tri, int n, float* __restrict__ B, int* __restrict__ C) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float4 a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
  Box6 r;
  r.lo[0] = fminf(fminf(a.x, b.x), c.x);
  r.lo[1] = fminf(fminf(a.y, b.y), c.y);
  r.lo[2] = fminf(fminf(a.z, b.z), c.z);
  r.hi[0] = fmaxf(fmaxf(a.x, b.x), c.x);
  r.hi[1] = fmaxf(fmaxf(a.y, b.y), c.y);
  r.hi[2] = fmaxf(fmaxf(a.z, b.z), c.z);
  store_box(B, i, r);
  C[i] = i | 0x80000000;
}

// Nearest neighbour of every cluster within the window (least merged area,
// ties to the lower index).
__global__ void k_ploc_nn(const float* __restrict__ B, int m, int* __restrict__ N) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const Box6 bi = load_box(B, i);
  int best = -1;
  float ba = 3.4e38f;
  const int j0 = i - kPlocRadius < 0 ? 0 : i - kPlocRadius;
  const int j1 = i + kPlocRadius > m - 1 ? m - 1 : i + kPlocRadius;
  for (int j = j0; j <= j1; ++j) {
    if (j == i) continue;
    const float a = half_area_rn(box_union(bi, load_box(B, j)));
    if (a < ba || (a == ba && j < best)) {
      ba = a;
      best = j;
    }
  }
  N[i] = best;
}

// Flags: bit 0 = i merges with its (higher-index) mutual neighbour, bit 1 =
// i survives compaction (it is not the higher index of a mutual pair).
__global__ void k_ploc_flags(const int* __restrict__ N, int m, int2* __restrict__ F) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int j = N[i];
  const bool mutual = j >= 0 && N[j] == i;
  F[i] = make_int2((mutual && i < j) ? 1 : 0, (mutual && j < i) ? 0 : 1);
}

// Exclusive scan of the flag pairs with one block (m up to a few million):
// each thread sums a contiguous chunk, the block scans the partial sums,
// then each thread writes its chunk's prefixes.  totals = (merges, survivors).
__global__ void k_scan_pairs(const int2* __restrict__ F, int m, int2* __restrict__ S, int2* __restrict__ totals) {
  __shared__ int2 part[1024];
  const int t = threadIdx.x;
  const int chunk = (m + blockDim.x - 1) / blockDim.x;
  const int b = t * chunk, e = min(m, b + chunk);
  int2 acc = make_int2(0, 0);
  for (int i = b; i < e; ++i) {
    acc.x += F[i].x;
    acc.y += F[i].y;
  }
  part[t] = acc;
  __syncthreads();
  for (int off = 1; off < (int)blockDim.x; off <<= 1) {
    int2 v = t >= off ? part[t - off] : make_int2(0, 0);
    __syncthreads();
    part[t].x += v.x;
    part[t].y += v.y;
    __syncthreads();
  }
  int2 run = t > 0 ? part[t - 1] : make_int2(0, 0);
  for (int i = b; i < e; ++i) {
    S[i] = run;
    run.x += F[i].x;
    run.y += F[i].y;
  }
  if (t == (int)blockDim.x - 1) *totals = part[t];
}

// Merge mutual pairs into new nodes (index (n-2) - creation order, so the
// root, created last, is node 0) and compact the clusters in order.
__global__ void k_ploc_apply(const float* __restrict__ B, const int* __restrict__ C, const int* __restrict__ N,
                             const int2* __restrict__ F, const int2* __restrict__ S, int m, int n, int created,
                             float* __restrict__ B2, int* __restrict__ C2, float* __restrict__ nodes) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int2 f = F[i];
  if (!f.y) return;
  const int2 pos = S[i];
  const Box6 bi = load_box(B, i);
  if (f.x) {
    const int j = N[i];
    const Box6 bj = load_box(B, j);
    const int x = (n - 2) - (created + pos.x);
    float* Nd = nodes + 16 * x;
    for (int k = 0; k < 3; ++k) {
      Nd[k] = bi.lo[k];
      Nd[3 + k] = bi.hi[k];
      Nd[6 + k] = bj.lo[k];
      Nd[9 + k] = bj.hi[k];
    }
    Nd[12] = __int_as_float(C[i]);
    Nd[13] = __int_as_float(C[j]);
    Nd[14] = 0.0f;
    Nd[15] = 0.0f;
    store_box(B2, pos.y, box_union(bi, bj));
    C2[pos.y] = x;
  } else {
    store_box(B2, pos.y, bi);
    C2[pos.y] = C[i];
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
  float* Bb = nullptr;
  int *Cb = nullptr, *Nn = nullptr;
  int2 *Fl = nullptr, *Sc = nullptr, *Tot = nullptr;
  cudaError_t e = cudaSuccess;
#define GR_TRY(x)                 \
  do {                            \
    e = (x);                      \
    if (e != cudaSuccess) goto done; \
  } while (0)
  GR_TRY(cudaMallocAsync(&cen, sizeof(float4) * n, st));
  GR_TRY(cudaMallocAsync(&b6, sizeof(float) * 6, st));
  GR_TRY(cudaMallocAsync(&keys, sizeof(unsigned long long) * n_pad, st));
  k_centroids<<<(n + 255) / 256, 256, 0, st>>>(verts, n, cen);
  k_bounds<<<1, 1024, 0, st>>>(cen, n, b6);
  k_morton<<<(n_pad + 255) / 256, 256, 0, st>>>(cen, n, n_pad, b6, keys);
  GR_TRY(cudaGetLastError());
  GR_TRY(launch_sort(keys, n_pad, st));
  k_reorder<<<(n + 255) / 256, 256, 0, st>>>(keys, n, verts, tri_mat, tri, tmat);
  GR_TRY(cudaGetLastError());
  if (n > 1) {
    GR_TRY(cudaMallocAsync(&Bb, sizeof(float) * 6 * 2 * (size_t)n, st));
    GR_TRY(cudaMallocAsync(&Cb, sizeof(int) * 2 * (size_t)n, st));
    GR_TRY(cudaMallocAsync(&Nn, sizeof(int) * (size_t)n, st));
    GR_TRY(cudaMallocAsync(&Fl, sizeof(int2) * (size_t)n, st));
    GR_TRY(cudaMallocAsync(&Sc, sizeof(int2) * (size_t)n, st));
    GR_TRY(cudaMallocAsync(&Tot, sizeof(int2), st));
    float* Bc = Bb;
    float* Bn = Bb + 6 * (size_t)n;
    int* Cc = Cb;
    int* Cn = Cb + n;
    k_leaf_clusters<<<(n + 255) / 256, 256, 0, st>>>(tri, n, Bc, Cc);
    int m = n, created = 0;
    for (int it = 0; m > 1 && it < n; ++it) {
      const int g = (m + 255) / 256;
      k_ploc_nn<<<g, 256, 0, st>>>(Bc, m, Nn);
      k_ploc_flags<<<g, 256, 0, st>>>(Nn, m, Fl);
      k_scan_pairs<<<1, 1024, 0, st>>>(Fl, m, Sc, Tot);
      k_ploc_apply<<<g, 256, 0, st>>>(Bc, Cc, Nn, Fl, Sc, m, n, created, Bn, Cn, nodes);
      int2 tot;
      GR_TRY(cudaMemcpyAsync(&tot, Tot, sizeof tot, cudaMemcpyDeviceToHost, st));
      GR_TRY(cudaStreamSynchronize(st));
      created += tot.x;
      m = tot.y;
      std::swap(Bc, Bn);
      std::swap(Cc, Cn);
    }
    if (m != 1 || created != n - 1) {
      e = cudaErrorUnknown;
      goto done;
    }
  }
  if (keys_out) GR_TRY(cudaMemcpyAsync(keys_out, keys, sizeof(unsigned long long) * n, cudaMemcpyDeviceToDevice, st));
done:
  if (cen) cudaFreeAsync(cen, st);
  if (b6) cudaFreeAsync(b6, st);
  if (keys) cudaFreeAsync(keys, st);
  if (Bb) cudaFreeAsync(Bb, st);
  if (Cb) cudaFreeAsync(Cb, st);
  if (Nn) cudaFreeAsync(Nn, st);
  if (Fl) cudaFreeAsync(Fl, st);
  if (Sc) cudaFreeAsync(Sc, st);
  if (Tot) cudaFreeAsync(Tot, st);
#undef GR_TRY
  return e;
}

// ------------------------------------------------------------------ 4-wide quantised BVH
// Derived from the binary LBVH: each wide node takes a binary node and expands
// its largest-area internal child until it has up to four children.  A wide
// node stores its box origin P (float32), one power-of-two scale 2^e per axis
// and 8-bit child bounds q with  P + qlo 2^e <= child lo  and  P + qhi 2^e >=
// child hi, computed in FP64 from exact float32 values, so every decoded box
// contains its child: the traversal can only visit more, never miss a hit.
// Layout (64 bytes = 4 x uint4):
//   w0..2 P.xyz, w3 = e.x | e.y << 8 | e.z << 16 (biased by 128) | count << 24
//   w4..9 child bytes: qlo.x[4], qlo.y[4], qlo.z[4], qhi.x[4], qhi.y[4], qhi.z[4]
//   w10..13 child references (bit 31 set = leaf slot; -1 = empty)
//   w14..15 unused

namespace {

struct BoxF {
  float lo[3], hi[3];
};

__device__ __forceinline__ BoxF leaf_box(const float4* tri, int slot) {
  const float4 a = tri[3 * slot], b = tri[3 * slot + 1], c = tri[3 * slot + 2];
  BoxF r;
  r.lo[0] = fminf(fminf(a.x, b.x), c.x);
  r.lo[1] = fminf(fminf(a.y, b.y), c.y);
  r.lo[2] = fminf(fminf(a.z, b.z), c.z);
  r.hi[0] = fmaxf(fmaxf(a.x, b.x), c.x);
  r.hi[1] = fmaxf(fmaxf(a.y, b.y), c.y);
  r.hi[2] = fmaxf(fmaxf(a.z, b.z), c.z);
  return r;
}

// Box of every binary internal node (from its parent's child-box slots).
__global__ void k_node_boxes(const float* __restrict__ nodes, int n, float* __restrict__ nbox) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const float* N = nodes + 16 * i;
  const int l = __float_as_int(N[12]), r = __float_as_int(N[13]);
  if (l >= 0)
    for (int k = 0; k < 6; ++k) nbox[6 * l + k] = N[k];
  if (r >= 0)
    for (int k = 0; k < 6; ++k) nbox[6 * r + k] = N[6 + k];
  if (i == 0)
    for (int k = 0; k < 3; ++k) {
      nbox[k] = fminf(N[k], N[6 + k]);
      nbox[3 + k] = fmaxf(N[3 + k], N[9 + k]);
    }
}

__device__ __forceinline__ BoxF ref_box(int ref, const float* nbox, const float4* tri) {
  if (ref < 0) return leaf_box(tri, ref & 0x7fffffff);
  BoxF b;
  for (int k = 0; k < 3; ++k) {
    b.lo[k] = nbox[6 * ref + k];
    b.hi[k] = nbox[6 * ref + 3 + k];
  }
  return b;
}

__device__ __forceinline__ float half_area(const BoxF& b) {
  const float dx = b.hi[0] - b.lo[0], dy = b.hi[1] - b.lo[1], dz = b.hi[2] - b.lo[2];
  return dx * dy + dy * dz + dz * dx;
}

// One level of the top-down collapse: frontier item (binary node, wide index).
__global__ void k_collapse(const float* __restrict__ nodes, const float* __restrict__ nbox,
                           const float4* __restrict__ tri, const int2* __restrict__ front, int n_front,
                           int2* __restrict__ next, int* __restrict__ counters, uint4* __restrict__ wn) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_front) return;
  const int bnode = front[t].x, widx = front[t].y;
  int ch[4];
  int cnt = 2;
  ch[0] = __float_as_int(nodes[16 * bnode + 12]);
  ch[1] = __float_as_int(nodes[16 * bnode + 13]);
  while (cnt < 4) {
    int best = -1;
    float ba = -1.0f;
    for (int k = 0; k < cnt; ++k)
      if (ch[k] >= 0) {
        float a = half_area(ref_box(ch[k], nbox, tri));
        if (a > ba) {
          ba = a;
          best = k;
        }
      }
    if (best < 0) break;
    const int x = ch[best];
    ch[best] = __float_as_int(nodes[16 * x + 12]);
    ch[cnt++] = __float_as_int(nodes[16 * x + 13]);
  }
  BoxF cb[4];
  BoxF W;
  for (int k = 0; k < 3; ++k) {
    W.lo[k] = 3.4e38f;
    W.hi[k] = -3.4e38f;
  }
  for (int c = 0; c < cnt; ++c) {
    cb[c] = ref_box(ch[c], nbox, tri);
    for (int k = 0; k < 3; ++k) {
      W.lo[k] = fminf(W.lo[k], cb[c].lo[k]);
      W.hi[k] = fmaxf(W.hi[k], cb[c].hi[k]);
    }
  }
  unsigned char qlo[3][4], qhi[3][4];
  int ex[3];
  for (int k = 0; k < 3; ++k) {
    const double ext = (double)W.hi[k] - (double)W.lo[k];
    int e = -100;
    if (ext > 0.0) {
      e = (int)ceil(log2(ext / 255.0));
      while (ldexp(255.0, e) < ext) ++e;
      if (e < -100) e = -100;
    }
    ex[k] = e;
    const double sc = ldexp(1.0, e);
    for (int c = 0; c < 4; ++c) {
      if (c < cnt) {
        double lo = floor(((double)cb[c].lo[k] - (double)W.lo[k]) / sc);
        double hi = ceil(((double)cb[c].hi[k] - (double)W.lo[k]) / sc);
        lo = lo < 0.0 ? 0.0 : (lo > 255.0 ? 255.0 : lo);
        hi = hi < 0.0 ? 0.0 : (hi > 255.0 ? 255.0 : hi);
        qlo[k][c] = (unsigned char)lo;
        qhi[k][c] = (unsigned char)hi;
      } else {
        qlo[k][c] = 255;  // empty slot: an inverted box that no ray hits
        qhi[k][c] = 0;
      }
    }
  }
  int refs[4] = {-1, -1, -1, -1};
  for (int c = 0; c < cnt; ++c) {
    if (ch[c] < 0) {
      refs[c] = ch[c];
    } else {
      const int w = atomicAdd(counters + 0, 1);
      refs[c] = w;
      const int f = atomicAdd(counters + 1, 1);
      next[f] = make_int2(ch[c], w);
    }
  }
  uint4 a, b, c4, d;
  a.x = __float_as_uint(W.lo[0]);
  a.y = __float_as_uint(W.lo[1]);
  a.z = __float_as_uint(W.lo[2]);
  a.w = (unsigned)(ex[0] + 128) | ((unsigned)(ex[1] + 128) << 8) | ((unsigned)(ex[2] + 128) << 16) |
        ((unsigned)cnt << 24);
  auto pack4 = [](const unsigned char* v) {
    return (unsigned)v[0] | ((unsigned)v[1] << 8) | ((unsigned)v[2] << 16) | ((unsigned)v[3] << 24);
  };
  b.x = pack4(qlo[0]);
  b.y = pack4(qlo[1]);
  b.z = pack4(qlo[2]);
  b.w = pack4(qhi[0]);
  c4.x = pack4(qhi[1]);
  c4.y = pack4(qhi[2]);
  c4.z = (unsigned)refs[0];
  c4.w = (unsigned)refs[1];
  d.x = (unsigned)refs[2];
  d.y = (unsigned)refs[3];
  d.z = 0u;
  d.w = 0u;
  wn[4 * widx] = a;
  wn[4 * widx + 1] = b;
  wn[4 * widx + 2] = c4;
  wn[4 * widx + 3] = d;
}

// 32-byte binary nodes: the two child boxes of node i in FP16, each lower
// bound rounded toward -inf and each upper bound toward +inf (so the FP16 box
// contains the FP32 one; values beyond the FP16 range become +-inf or the
// largest finite value on the safe side), then the two child references.
// Halves: [l.lo.x l.lo.y][l.lo.z l.hi.x][l.hi.y l.hi.z][r.lo.x r.lo.y]
// [r.lo.z r.hi.x][r.hi.y r.hi.z], low half of each word first.  Node i is
// stored at position pos[i] and its internal child references are renumbered
// the same way (leaf references are triangle slots and stay).
__global__ void k_half_nodes(const float* __restrict__ nodes, int n, const int* __restrict__ pos,
                             uint4* __restrict__ hn) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n - 1) return;
  const float* N = nodes + 16 * (size_t)i;
  unsigned short h[12];
  for (int c = 0; c < 2; ++c)
    for (int a = 0; a < 3; ++a) {
      h[6 * c + a] = __half_as_ushort(__float2half_rd(N[6 * c + a]));
      h[6 * c + 3 + a] = __half_as_ushort(__float2half_ru(N[6 * c + 3 + a]));
    }
  uint4 q0, q1;
  q0.x = (unsigned)h[0] | ((unsigned)h[1] << 16);
  q0.y = (unsigned)h[2] | ((unsigned)h[3] << 16);
  q0.z = (unsigned)h[4] | ((unsigned)h[5] << 16);
  q0.w = (unsigned)h[6] | ((unsigned)h[7] << 16);
  q1.x = (unsigned)h[8] | ((unsigned)h[9] << 16);
  q1.y = (unsigned)h[10] | ((unsigned)h[11] << 16);
  const int l = __float_as_int(N[12]), r = __float_as_int(N[13]);
  q1.z = (unsigned)(l >= 0 ? pos[l] : l);
  q1.w = (unsigned)(r >= 0 ? pos[r] : r);
  const size_t d = (size_t)pos[i];
  hn[2 * d] = q0;
  hn[2 * d + 1] = q1;
}

}  // namespace

// FP16 copy of the binary nodes (n >= 2 leaves): hn holds (n - 1) x 32 bytes,
// in depth-first order from the root (left child first), so that a node and
// its left internal child are neighbours in memory and a subtree occupies one
// contiguous range: a traversal's consecutive node fetches then often fall in
// a cache line already read.  The order is computed on the host from the
// nodes' child references (8 bytes per node copied back), before the
// conversion kernel writes each node at its new position.  The tree, its
// boxes and its closest hits are those of the FP32 nodes.
cudaError_t build_half(const float* nodes, int n, uint4* hn, cudaStream_t st) {
  if (n < 2) return cudaSuccess;
  const int m = n - 1;
  std::vector<int2> refs((size_t)m);
  cudaError_t e = cudaMemcpy2DAsync(refs.data(), sizeof(int2), nodes + 12, 16 * sizeof(float), sizeof(int2), (size_t)m,
                                    cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  std::vector<int> pos((size_t)m, -1), stack;
  stack.reserve(128);
  stack.push_back(0);
  int next = 0;
  while (!stack.empty()) {
    const int x = stack.back();
    stack.pop_back();
    // a malformed tree (a node reached twice, an index out of range) keeps
    // the identity order; the traversal's own bounds then report it
    if (x < 0 || x >= m || pos[(size_t)x] >= 0 || next >= m) {
      next = -1;
      break;
    }
    pos[(size_t)x] = next++;
    const int2 c = refs[(size_t)x];
    if (c.y >= 0) stack.push_back(c.y);
    if (c.x >= 0) stack.push_back(c.x);
  }
  if (next != m)
    for (int i = 0; i < m; ++i) pos[(size_t)i] = i;
  int* pos_d = nullptr;
  e = cudaMallocAsync(&pos_d, sizeof(int) * (size_t)m, st);
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(pos_d, pos.data(), sizeof(int) * (size_t)m, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_half_nodes<<<(m + 255) / 256, 256, 0, st>>>(nodes, n, pos_d, hn);
    e = cudaGetLastError();
  }
  // the host order must outlive its copy
  const cudaError_t e2 = cudaStreamSynchronize(st);
  cudaFreeAsync(pos_d, st);
  return e != cudaSuccess ? e : e2;
}

// Collapse the binary LBVH (n >= 2 leaves) into 4-wide quantised nodes.  wn
// must hold (n - 1) nodes (an upper bound); *n_wide receives the count.
cudaError_t build_wide(const float* nodes, const float4* tri, int n, uint4* wn, int* n_wide, cudaStream_t st) {
  *n_wide = 0;
  if (n < 2) return cudaSuccess;
  float* nbox = nullptr;
  int2 *fa = nullptr, *fb = nullptr;
  int* ctr = nullptr;
  cudaError_t e = cudaSuccess;
  int h_ctr[2];
  int n_front = 1;
  int2 root = make_int2(0, 0);
  if ((e = cudaMallocAsync(&nbox, sizeof(float) * 6 * (size_t)(n - 1), st)) != cudaSuccess) goto out;
  if ((e = cudaMallocAsync(&fa, sizeof(int2) * (size_t)n, st)) != cudaSuccess) goto out;
  if ((e = cudaMallocAsync(&fb, sizeof(int2) * (size_t)n, st)) != cudaSuccess) goto out;
  if ((e = cudaMallocAsync(&ctr, sizeof(int) * 2, st)) != cudaSuccess) goto out;
  k_node_boxes<<<(n - 1 + 255) / 256, 256, 0, st>>>(nodes, n, nbox);
  if ((e = cudaMemcpyAsync(fa, &root, sizeof root, cudaMemcpyHostToDevice, st)) != cudaSuccess) goto out;
  h_ctr[0] = 1;  // wide node 0 is the root
  h_ctr[1] = 0;
  if ((e = cudaMemcpyAsync(ctr, h_ctr, sizeof h_ctr, cudaMemcpyHostToDevice, st)) != cudaSuccess) goto out;
  for (int level = 0; level < 4 * 64 && n_front > 0; ++level) {
    k_collapse<<<(n_front + 127) / 128, 128, 0, st>>>(nodes, nbox, tri, fa, n_front, fb, ctr, wn);
    if ((e = cudaMemcpyAsync(h_ctr, ctr, sizeof h_ctr, cudaMemcpyDeviceToHost, st)) != cudaSuccess) goto out;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) goto out;
    n_front = h_ctr[1];
    h_ctr[1] = 0;
    if ((e = cudaMemcpyAsync(ctr + 1, &h_ctr[1], sizeof(int), cudaMemcpyHostToDevice, st)) != cudaSuccess) goto out;
    int2* t = fa;
    fa = fb;
    fb = t;
  }
  *n_wide = h_ctr[0];
  e = cudaGetLastError();
out:
  if (nbox) cudaFreeAsync(nbox, st);
  if (fa) cudaFreeAsync(fa, st);
  if (fb) cudaFreeAsync(fb, st);
  if (ctr) cudaFreeAsync(ctr, st);
  return e;
}

}  // namespace gr
