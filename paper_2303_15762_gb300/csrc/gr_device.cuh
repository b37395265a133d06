// Device-side building blocks of the generalized-ray path tracer (sm_103a).
// Everything on the render path is FP32 except the decision refinements and the
// footprint quadratic form at emitters, which run in FP64.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "gr.h"

namespace gr {

constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;
// Hits closer than this (metres) are ignored, besides the primitive just left.
constexpr float kTMin = 1e-5f;
// Roughness above which the Poisson series is replaced by its continuous limit.
constexpr float kGCont = 50.0f;
// Largest grating order magnitude kept in the order tables.
constexpr int kMaxOrder = 40;
constexpr int kStackDepth = 64;
// BVH layouts a traversal can walk: the binary tree with FP32 child boxes (64
// bytes per node), the same tree with FP16 child boxes rounded outward (32
// bytes per node, the default), or the 4-wide tree with 8-bit child boxes.
enum Tree { kTreeF32 = 0, kTreeWide = 1, kTreeHalf = 2 };

// Random-number uses at a path vertex (word 2 of the Philox counter is
// (segment << 4) | call).
enum Call { kCallJitter = 0, kCallEmitFoot = 1, kCallLobe = 2, kCallNeeDir = 3, kCallNeeFoot = 4, kCallRR = 5 };

// ------------------------------------------------------------------ device scene
struct DevEmitter {
  int mat;       // emitter material id
  int first;     // first triangle in emitter_tris
  int count;     // number of triangles
  int planar;    // 1 if every triangle lies in the first one's plane
  float lo[3];   // bounding box of the emitter's triangles
  float hi[3];
  float n[3];    // unit normal of the first triangle (front face), FP32
  int pad;
  double nd[3];  // the same normal in FP64 (for the measurement lobe's quadratic form)
};

struct DevScene {
  int n_tris;
  int n_mats;
  int n_lights;
  int n_emitters;
  const float4* tri;         // [n][3] vertices in BVH leaf order; tri[3i].w = original id (int bits)
  const int* tri_mat;        // [n] material of leaf slot i
  const float4* nodes;       // [n-1][4] internal nodes (child boxes + child refs)
  const uint4* wnodes;       // [n_wide][4] 4-wide quantised nodes (root = 0)
  const uint4* hnodes;       // [n-1][2] the binary nodes with FP16 child boxes rounded outward (32 bytes),
                             // or null when the scene's coordinates exceed the FP16 range
  int n_wide;
  int pad_w;
  const gr_material* mats;   // [n_mats]
  const gr_light* lights;    // [n_lights]
  const DevEmitter* emitters;     // [n_emitters]
  const int* emitter_of_mat;      // [n_mats] -> emitter index or -1
  const float4* emitter_tris;     // [m][3] vertices of emitter triangles
};

struct DevView {
  float3 eye, fw, right, upc;
  float th, aspect;
  int W, H, nb, ns, max_depth, spp, first_sample, view_index, scene_index, ortho;
  float ortho_half;
  float lmin, lmax, beta0;
  long long ticket_base;  // first global ticket of this view
  long long n_tickets;    // nbu * W * H
  float* acc_sum;         // [nb][H][W][ns]
  float* acc_comp;
  int table_base;         // first table row of this view ((view, material, bin) rows)
  int nbu;                // sample classes that receive samples: min(spp, Q), from first_sample mod Q on
  int Q;                  // class modulus: a ticket owns the samples s with s mod Q == its class
                          // (Q = nb: one bin per ticket; Q = nb/4 with hero-wavelength MIS)
  int hs;                 // hero-wavelength MIS: tickets per class (its samples in hs
                          // consecutive ranges, combined in range order); 1 otherwise
  long long hbase;        // first class record of this view in the range-sum buffer (hs > 1)
};

// Per-(view, material, bin) row of the grating order table: J_j(h k/2)^2 for
// j = 0..jmax, stored from `offset` in the value array.
struct TableRow {
  int offset;
  int jmax;
};

// ------------------------------------------------------------------ small vector math
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(s * a.x, s * a.y, s * a.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float dot(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize(float3 a) { return rsqrtf(dot(a, a)) * a; }
__device__ __forceinline__ float3 xyz(float4 a) { return f3(a.x, a.y, a.z); }

struct d3 {
  double x, y, z;
};
__device__ __forceinline__ d3 D3(float3 a) { return d3{a.x, a.y, a.z}; }
__device__ __forceinline__ d3 dadd(d3 a, d3 b) { return d3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ d3 dsub(d3 a, d3 b) { return d3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ d3 dmul(double s, d3 a) { return d3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double ddot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ d3 dcross(d3 a, d3 b) {
  return d3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ d3 dnormalize(d3 a) { return dmul(1.0 / sqrt(ddot(a, a)), a); }

// Branchless orthonormal basis (Duff et al., JCGT 2017).
__device__ __forceinline__ void onb(float3 n, float3& e1, float3& e2) {
  float sign = copysignf(1.0f, n.z);
  float a = -1.0f / (sign + n.z);
  float b = n.x * n.y * a;
  e1 = f3(1.0f + sign * n.x * n.x * a, sign * b, -sign * n.x);
  e2 = f3(b, sign + n.y * n.y * a, -n.y);
}
__device__ __forceinline__ void onb_d(d3 n, d3& e1, d3& e2) {
  double sign = copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  e1 = d3{1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x};
  e2 = d3{b, sign + n.y * n.y * a, -n.y};
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon et al., SC'11: 10 rounds; multipliers 0xD2511F53 / 0xCD9E8D57, key
// schedule 0x9E3779B9 / 0xBB67AE85, applied between rounds.
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// Four uniforms in [0,1) on the 2^-24 grid for (pixel, sample, segment, call).
__device__ __forceinline__ float4 rng4(uint32_t seed, uint32_t view, uint32_t pixel, uint32_t sample, int seg,
                                       int call) {
  uint4 x = philox10(make_uint4(pixel, sample, ((uint32_t)seg << 4) | (uint32_t)call, 0u), seed, view);
  const float s = 5.9604644775390625e-8f;  // 2^-24
  return make_float4((float)(x.x >> 8) * s, (float)(x.y >> 8) * s, (float)(x.z >> 8) * s, (float)(x.w >> 8) * s);
}

__device__ __forceinline__ void box_muller(float u0, float u1, float& z0, float& z1) {
  float r = sqrtf(-2.0f * logf(1.0f - u0));
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  z0 = r * c;
  z1 = r * s;
}

// vMF density about mu with concentration kappa (angular Gaussian on the sphere).
__device__ __forceinline__ float vmf(float3 w, float3 mu, float kappa) {
  if (kappa < 1e-8f) return 0.25f / kPi;
  float3 d = w - mu;
  return kappa / (2.0f * kPi * (-expm1f(-2.0f * kappa))) * expf(-0.5f * kappa * dot(d, d));
}
__device__ __forceinline__ double vmf_d(d3 w, d3 mu, double kappa) {
  if (kappa < 1e-8) return 0.25 / kPiD;
  d3 d = dsub(w, mu);
  return kappa / (2.0 * kPiD * (-expm1(-2.0 * kappa))) * exp(-0.5 * kappa * ddot(d, d));
}

__device__ __forceinline__ float3 vmf_sample(float3 mu, float kappa, float u0, float u1) {
  float up = 1.0f - u0;
  float v = -logf(up + (1.0f - up) * expf(-2.0f * kappa)) / kappa;  // 1 - cos(theta)
  float sin_t = sqrtf(fmaxf(0.0f, v * (2.0f - v)));
  float s, c;
  sincospif(2.0f * u1, &s, &c);
  float3 e1, e2;
  onb(mu, e1, e2);
  return normalize((sin_t * c) * e1 + (sin_t * s) * e2 + (1.0f - v) * mu);
}

// ------------------------------------------------------------------ Bessel J_n (power series)
__device__ __forceinline__ double bessel_j_d(int n, double x) {
  if (n < 0) n = -n;  // only squares are used
  double half = 0.5 * x, term = 1.0;
  for (int i = 1; i <= n; ++i) term *= half / i;
  double sum = term;
  for (int m = 1; m < 200; ++m) {
    term *= -(half * half) / ((double)m * (double)(m + n));
    sum += term;
    if (fabs(term) < 1e-18 * fabs(sum) && m > 2) break;
  }
  return sum;
}

// ------------------------------------------------------------------ intersection
struct RayPre {
  float3 o, d, inv;
  int kx, ky, kz;
  float Sx, Sy, Sz;
};

__device__ __forceinline__ float comp(float3 v, int i) { return i == 0 ? v.x : (i == 1 ? v.y : v.z); }

__device__ __forceinline__ RayPre ray_pre(float3 o, float3 d) {
  RayPre r;
  r.o = o;
  r.d = d;
  r.inv = f3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
  float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
  int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
  int kx = kz + 1 == 3 ? 0 : kz + 1;
  int ky = kx + 1 == 3 ? 0 : kx + 1;
  if (comp(d, kz) < 0.0f) {
    int t = kx;
    kx = ky;
    ky = t;
  }
  r.kx = kx;
  r.ky = ky;
  r.kz = kz;
  float dz = comp(d, kz);
  r.Sx = comp(d, kx) / dz;
  r.Sy = comp(d, ky) / dz;
  r.Sz = 1.0f / dz;
  return r;
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2(1), 2013) in FP32.
// When an edge function lies within its FP32 rounding bound the three edge
// functions are recomputed in FP64 from the same FP32 inputs ("FP64
// refinement"), so the inside/outside decision is exact for the ray as stored.
// The bound: the sheared coordinates carry an absolute error of a few ulps of
// the largest vertex offset M, so |dU| <= c * u * M * (|Bx|+|By|+|Cx|+|Cy|) plus
// the rounding of the products themselves.  Edges count as inside.
// Returns t (metres) or -1; *refined counts FP64 recomputations.
__device__ __forceinline__ float isect_tri(const RayPre& r, float3 v0, float3 v1, float3 v2, int* refined) {
  const float3 A = v0 - r.o, B = v1 - r.o, C = v2 - r.o;
  const float Az_ = comp(A, r.kz), Bz_ = comp(B, r.kz), Cz_ = comp(C, r.kz);
  const float Ax = comp(A, r.kx) - r.Sx * Az_, Ay = comp(A, r.ky) - r.Sy * Az_;
  const float Bx = comp(B, r.kx) - r.Sx * Bz_, By = comp(B, r.ky) - r.Sy * Bz_;
  const float Cx = comp(C, r.kx) - r.Sx * Cz_, Cy = comp(C, r.ky) - r.Sy * Cz_;
  float U = Cx * By - Cy * Bx;
  float V = Ax * Cy - Ay * Cx;
  float W = Bx * Ay - By * Ax;
  const float M = fmaxf(fmaxf(fmaxf(fabsf(A.x), fabsf(A.y)), fmaxf(fabsf(A.z), fabsf(B.x))),
                        fmaxf(fmaxf(fabsf(B.y), fabsf(B.z)), fmaxf(fmaxf(fabsf(C.x), fabsf(C.y)), fabsf(C.z))));
  const float e = 8.0f * 5.9604645e-8f * M * (1.0f + fabsf(r.Sx) + fabsf(r.Sy));
  const bool refine = fabsf(U) <= e * (fabsf(Bx) + fabsf(By) + fabsf(Cx) + fabsf(Cy)) + 4e-7f * (fabsf(Cx * By) + fabsf(Cy * Bx)) ||
                      fabsf(V) <= e * (fabsf(Ax) + fabsf(Ay) + fabsf(Cx) + fabsf(Cy)) + 4e-7f * (fabsf(Ax * Cy) + fabsf(Ay * Cx)) ||
                      fabsf(W) <= e * (fabsf(Ax) + fabsf(Ay) + fabsf(Bx) + fabsf(By)) + 4e-7f * (fabsf(Bx * Ay) + fabsf(By * Ax));
  if (refine) {
    // FP64 edge functions from the FP32 vertices and ray
    const double dz = (double)comp(r.d, r.kz);
    const double Sx = (double)comp(r.d, r.kx) / dz;
    const double Sy = (double)comp(r.d, r.ky) / dz;
    const d3 o = D3(r.o);
    const d3 a = dsub(D3(v0), o), b = dsub(D3(v1), o), c = dsub(D3(v2), o);
    auto cm = [&](d3 v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); };
    const double ax = cm(a, r.kx) - Sx * cm(a, r.kz), ay = cm(a, r.ky) - Sy * cm(a, r.kz);
    const double bx = cm(b, r.kx) - Sx * cm(b, r.kz), by = cm(b, r.ky) - Sy * cm(b, r.kz);
    const double cx = cm(c, r.kx) - Sx * cm(c, r.kz), cy = cm(c, r.ky) - Sy * cm(c, r.kz);
    const double Ud = cx * by - cy * bx, Vd = ax * cy - ay * cx, Wd = bx * ay - by * ax;
    // keep the exact signs; magnitudes only feed t below
    U = Ud == 0.0 ? 0.0f : (fabs(Ud) < 1e-37 ? copysignf(1e-37f, (float)Ud) : (float)Ud);
    V = Vd == 0.0 ? 0.0f : (fabs(Vd) < 1e-37 ? copysignf(1e-37f, (float)Vd) : (float)Vd);
    W = Wd == 0.0 ? 0.0f : (fabs(Wd) < 1e-37 ? copysignf(1e-37f, (float)Wd) : (float)Wd);
    ++*refined;
  }
  if ((U < 0.0f || V < 0.0f || W < 0.0f) && (U > 0.0f || V > 0.0f || W > 0.0f)) return -1.0f;
  const float det = U + V + W;
  if (det == 0.0f) return -1.0f;
  const float T = U * (r.Sz * Az_) + V * (r.Sz * Bz_) + W * (r.Sz * Cz_);
  return T / det;
}

// Slab test of a child box; returns the entry distance (>= 0), or -1 when the
// box is missed or starts beyond tbest.
// The far distance is widened by 2*gamma(3) (Ize 2013) so no box containing a
// triangle hit is rejected by rounding.
__device__ __forceinline__ float box_entry(const RayPre& r, float3 lo, float3 hi, float tbest) {
  float tx0 = (lo.x - r.o.x) * r.inv.x, tx1 = (hi.x - r.o.x) * r.inv.x;
  float ty0 = (lo.y - r.o.y) * r.inv.y, ty1 = (hi.y - r.o.y) * r.inv.y;
  float tz0 = (lo.z - r.o.z) * r.inv.z, tz1 = (hi.z - r.o.z) * r.inv.z;
  float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
  float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
  tf = fminf(tf * 1.0000004f, tbest);
  return tn <= tf ? tn : -1.0f;
}

struct Hit {
  float t;
  int slot;  // leaf slot (BVH order) or -1
};

// Resumable traversal of the binary BVH for one ray: the state a lane keeps
// between steps, so a warp can interleave rays that started at different
// times.  One step visits one internal node (two slab tests, leaf children
// tested at once) and picks the next node, nearer child first, the farther
// one pushed; the order of visits and tests per ray does not depend on how
// steps are scheduled, so neither does the result.
struct BinTrav {
  RayPre r;
  float t;       // closest accepted distance so far (+inf: none)
  int slot;      // leaf slot of that hit, or -1
  int best_id;   // its original triangle id (ties go to the lower id)
  int exclude;   // leaf slot never accepted (the surface the ray leaves)
  int node, sp, guard;
};

__device__ __forceinline__ void bin_leaf(const float4* __restrict__ tri, BinTrav& s, int leaf, int* refined,
                                         int* tests) {
  if (leaf == s.exclude) return;
  const float4 a = __ldg(&tri[3 * leaf]);
  const float4 b = __ldg(&tri[3 * leaf + 1]);
  const float4 c = __ldg(&tri[3 * leaf + 2]);
  ++*tests;
  const float t = isect_tri(s.r, xyz(a), xyz(b), xyz(c), refined);
  const int id = __float_as_int(a.w);
  if (t > kTMin && (t < s.t || (t == s.t && id < s.best_id))) {
    s.t = t;
    s.slot = leaf;
    s.best_id = id;
  }
}

// Starts a traversal; returns true if it is already complete (0 or 1 triangles).
__device__ __forceinline__ bool bin_begin(int n_tris, const float4* __restrict__ tri, BinTrav& s, float3 o, float3 d,
                                          int exclude, int* refined, int* tests) {
  s.t = __int_as_float(0x7f800000);
  s.slot = -1;
  s.best_id = 0x7fffffff;
  s.exclude = exclude;
  s.node = 0;
  s.sp = 0;
  // a binary tree of n leaves has n-1 internal nodes: a traversal never visits
  // more, so the bound only trips on a corrupt hierarchy
  s.guard = n_tris + 8;
  if (n_tris == 0) return true;
  s.r = ray_pre(o, d);
  if (n_tris == 1) {
    bin_leaf(tri, s, 0, refined, tests);
    return true;
  }
  return false;
}

// Two FP16 values packed in a 32-bit word (low half first), as floats.
__device__ __forceinline__ float2 half2_bits_to_float2(unsigned w) {
  __half2_raw r;
  r.x = (unsigned short)(w & 0xffffu);
  r.y = (unsigned short)(w >> 16);
  return __half22float2(__half2(r));
}

// One node visit (HALF: the 32-byte FP16 node array, else the 64-byte FP32
// one); returns true when the traversal is complete.  Leaf
// children whose boxes the ray enters go to leaf(slot), which tests them at
// once or queues them: the closest hit is the least (t, original id) over the
// tested triangles whatever the order of the tests, and a test only ever
// lowers s.t, so a queued test only delays culling.  *err = 2 if the visit
// bound trips, 1 if the stack would overflow (the traversal then drops the
// farther child).  `stack` holds kStackDepth entries, kept outside BinTrav so
// that the ray state stays in registers.
template <bool HALF, class LeafFn>
__device__ __forceinline__ bool bin_step(const void* __restrict__ nodes, BinTrav& s, int* stack, int* visits,
                                         int* err, LeafFn&& leaf) {
  if (--s.guard < 0) {
    if (err) *err = 2;
    return true;
  }
  ++*visits;
  float tl, tr;
  int lref, rref;
  if (HALF) {
    // 32-byte node: halves [l.lo.x l.lo.y][l.lo.z l.hi.x][l.hi.y l.hi.z]
    // [r.lo.x r.lo.y][r.lo.z r.hi.x][r.hi.y r.hi.z], then lref, rref; the
    // boxes contain the FP32 ones, so a box the FP32 tree enters is entered
    const uint4* N = (const uint4*)nodes + 2 * s.node;
    const uint4 q0 = __ldg(N), q1 = __ldg(N + 1);
    const float2 a = half2_bits_to_float2(q0.x), b = half2_bits_to_float2(q0.y), c = half2_bits_to_float2(q0.z);
    const float2 d = half2_bits_to_float2(q0.w), e = half2_bits_to_float2(q1.x), f = half2_bits_to_float2(q1.y);
    lref = (int)q1.z;
    rref = (int)q1.w;
    tl = box_entry(s.r, f3(a.x, a.y, b.x), f3(b.y, c.x, c.y), s.t);
    tr = box_entry(s.r, f3(d.x, d.y, e.x), f3(e.y, f.x, f.y), s.t);
  } else {
    const float4* N = (const float4*)nodes + 4 * s.node;
    const float4 n0 = __ldg(N), n1 = __ldg(N + 1), n2 = __ldg(N + 2), n3 = __ldg(N + 3);
    lref = __float_as_int(n3.x);
    rref = __float_as_int(n3.y);
    tl = box_entry(s.r, f3(n0.x, n0.y, n0.z), f3(n0.w, n1.x, n1.y), s.t);
    tr = box_entry(s.r, f3(n1.z, n1.w, n2.x), f3(n2.y, n2.z, n2.w), s.t);
  }
  bool hl = tl >= 0.0f, hr = tr >= 0.0f;
  // leaves go to `leaf`; internal children are descended/pushed
  if (hl && lref < 0) {
    leaf(lref & 0x7fffffff);
    hl = false;
  }
  if (hr && rref < 0) {
    leaf(rref & 0x7fffffff);
    hr = false;
  }
  int next = -1;
  if (hl && hr) {
    const int nearer = tl <= tr ? lref : rref;
    const int farther = tl <= tr ? rref : lref;
    if (s.sp < kStackDepth) {
      stack[s.sp++] = farther;
    } else if (err) {
      *err = 1;
    }
    next = nearer;
  } else if (hl) {
    next = lref;
  } else if (hr) {
    next = rref;
  }
  if (next < 0) {
    if (s.sp == 0) return true;
    next = stack[--s.sp];
  }
  s.node = next;
  return false;
}

// Closest hit along (o, d) with t > kTMin, skipping leaf slot `exclude`;
// equal distances resolve to the lower original triangle id.  Stack-based
// traversal of the binary BVH, nearer child first.  *err is set if the stack
// would overflow (the traversal then stops early).
template <bool HALF = false>
__device__ __forceinline__ Hit closest_hit(const DevScene& S, float3 o, float3 d, int exclude, int* refined,
                                           int* visits, int* tests, int* err) {
  BinTrav s;
  int stack[kStackDepth];
  if (!bin_begin(S.n_tris, S.tri, s, o, d, exclude, refined, tests)) {
    const float4* tri = S.tri;
    auto test_now = [&](int leaf) { bin_leaf(tri, s, leaf, refined, tests); };
    const void* nodes = HALF ? (const void*)S.hnodes : (const void*)S.nodes;
    while (!bin_step<HALF>(nodes, s, stack, visits, err, test_now)) {
    }
  }
  Hit h;
  h.t = s.t;
  h.slot = s.slot;
  return h;
}

// Closest hit through the 4-wide quantised BVH: same contract as closest_hit
// (t > kTMin, skip `exclude`, ties to the lower original id).  A node decodes
// its child slabs as t = q * (2^e / d) + (P - o) / d, one FMA per bound; the
// far distance is widened by 8 ulps and the near one narrowed, so rounding
// can only add visits.
__device__ __forceinline__ Hit closest_hit_wide(const DevScene& S, float3 o, float3 d, int exclude, int* refined,
                                                int* visits, int* tests, int* err) {
  Hit h;
  h.t = __int_as_float(0x7f800000);
  h.slot = -1;
  int best_id = 0x7fffffff;
  if (S.n_tris == 0) return h;
  RayPre r = ray_pre(o, d);
  auto test_leaf = [&](int slot) {
    if (slot == exclude) return;
    const float4 a = __ldg(&S.tri[3 * slot]);
    const float4 b = __ldg(&S.tri[3 * slot + 1]);
    const float4 c = __ldg(&S.tri[3 * slot + 2]);
    ++*tests;
    float t = isect_tri(r, xyz(a), xyz(b), xyz(c), refined);
    int id = __float_as_int(a.w);
    if (t > kTMin && (t < h.t || (t == h.t && id < best_id))) {
      h.t = t;
      h.slot = slot;
      best_id = id;
    }
  };
  if (S.n_tris == 1 || S.n_wide == 0) {
    test_leaf(0);
    return h;
  }
  int stack[kStackDepth];
  int sp = 0;
  int node = 0;
  int guard = S.n_tris + 8;
  for (;;) {
    if (--guard < 0) {
      if (err) *err = 2;
      break;
    }
    ++*visits;
    const uint4* N = S.wnodes + 4 * node;
    const uint4 a = __ldg(N), b = __ldg(N + 1), c = __ldg(N + 2), e4 = __ldg(N + 3);
    const int cnt = (int)(a.w >> 24);
    const float sx = __int_as_float((int)(((a.w & 0xffu) - 128u + 127u) << 23));
    const float sy = __int_as_float((int)((((a.w >> 8) & 0xffu) - 128u + 127u) << 23));
    const float sz = __int_as_float((int)((((a.w >> 16) & 0xffu) - 128u + 127u) << 23));
    const float Ax = sx * r.inv.x, Ay = sy * r.inv.y, Az = sz * r.inv.z;
    const float Bx = (__uint_as_float(a.x) - r.o.x) * r.inv.x;
    const float By = (__uint_as_float(a.y) - r.o.y) * r.inv.y;
    const float Bz = (__uint_as_float(a.z) - r.o.z) * r.inv.z;
    const int refs[4] = {(int)c.z, (int)c.w, (int)e4.x, (int)e4.y};
    const float kInf = __int_as_float(0x7f800000);
    // entry distance of each internal child hit (+inf otherwise), kept in
    // fixed registers; leaves are tested on the spot
    float tq[4] = {kInf, kInf, kInf, kInf};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if (k < cnt) {
        const unsigned sh = 8u * k;
        const float lx = (float)((b.x >> sh) & 0xffu), ly = (float)((b.y >> sh) & 0xffu), lz = (float)((b.z >> sh) & 0xffu);
        const float hx = (float)((b.w >> sh) & 0xffu), hy = (float)((c.x >> sh) & 0xffu), hz = (float)((c.y >> sh) & 0xffu);
        const float tx0 = fmaf(lx, Ax, Bx), tx1 = fmaf(hx, Ax, Bx);
        const float ty0 = fmaf(ly, Ay, By), ty1 = fmaf(hy, Ay, By);
        const float tz0 = fmaf(lz, Az, Bz), tz1 = fmaf(hz, Az, Bz);
        float tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
        float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fmaxf(tz0, tz1));
        tn *= 0.999999f;
        tf = fminf(tf * 1.000001f, h.t);
        if (tn <= tf) {
          if (refs[k] < 0)
            test_leaf(refs[k] & 0x7fffffff);
          else
            tq[k] = tn;
        }
      }
    }
    // order the four (distance, child) pairs with a sorting network
    float t0 = tq[0], t1 = tq[1], t2 = tq[2], t3 = tq[3];
    int r0 = refs[0], r1 = refs[1], r2 = refs[2], r3 = refs[3];
    auto cswap = [](float& ta, int& ra, float& tb, int& rb) {
      if (tb < ta) {
        float t = ta;
        ta = tb;
        tb = t;
        int q = ra;
        ra = rb;
        rb = q;
      }
    };
    cswap(t0, r0, t1, r1);
    cswap(t2, r2, t3, r3);
    cswap(t0, r0, t2, r2);
    cswap(t1, r1, t3, r3);
    cswap(t1, r1, t2, r2);
    // nearest next; the others pushed farthest first (skipping those now
    // beyond the best hit)
    // (+inf marks "not an internal hit"; it must not pass as <= h.t = +inf)
    int next = -1;
    if (t0 < kInf && t0 <= h.t) {
      next = r0;
      if (t3 < kInf && t3 <= h.t) {
        if (sp < kStackDepth) stack[sp++] = r3;
        else if (err) *err = 1;
      }
      if (t2 < kInf && t2 <= h.t) {
        if (sp < kStackDepth) stack[sp++] = r2;
        else if (err) *err = 1;
      }
      if (t1 < kInf && t1 <= h.t) {
        if (sp < kStackDepth) stack[sp++] = r1;
        else if (err) *err = 1;
      }
    }
    if (next < 0) {
      if (sp == 0) break;
      next = stack[--sp];
    }
    node = next;
  }
  return h;
}

// ------------------------------------------------------------------ small complex (FP32)
struct cf {
  float re, im;
};
__device__ __forceinline__ cf cadd(cf a, cf b) { return cf{a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ cf csub(cf a, cf b) { return cf{a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ cf cmul(cf a, cf b) { return cf{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
__device__ __forceinline__ cf cdiv(cf a, cf b) {
  float den = b.re * b.re + b.im * b.im;
  return cf{(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
__device__ __forceinline__ cf csqrt(cf z) {
  // principal square root
  float m = sqrtf(z.re * z.re + z.im * z.im);
  float re = sqrtf(fmaxf(0.0f, 0.5f * (m + z.re)));
  float im = copysignf(sqrtf(fmaxf(0.0f, 0.5f * (m - z.re))), z.im);
  return cf{re, im};
}

// Fresnel reflection of a smooth conductor (n = n_re + i n_im): Mueller
// entries of diag(r_s, r_p) in s-p frames: a = (|rs|^2+|rp|^2)/2,
// b = (|rs|^2-|rp|^2)/2, cr + i ci = rs conj(rp).
struct FresnelM {
  float a, b, cr, ci;
};
__device__ __forceinline__ FresnelM fresnel_conductor(float cos_i, float n_re, float n_im) {
  cf n{n_re, n_im};
  float sin2 = fmaxf(0.0f, 1.0f - cos_i * cos_i);
  cf n2 = cmul(n, n);
  cf ncos_t = csqrt(cf{n2.re - sin2, n2.im});
  cf cos_t = cdiv(ncos_t, n);
  cf ci{cos_i, 0.0f};
  cf rs = cdiv(csub(ci, ncos_t), cadd(ci, ncos_t));
  cf nci = cmul(n, ci);
  cf rp = cdiv(csub(nci, cos_t), cadd(nci, cos_t));
  float A = rs.re * rs.re + rs.im * rs.im, B = rp.re * rp.re + rp.im * rp.im;
  FresnelM m;
  m.a = 0.5f * (A + B);
  m.b = 0.5f * (A - B);
  m.cr = rs.re * rp.re + rs.im * rp.im;   // Re(rs conj(rp))
  m.ci = rs.im * rp.re - rs.re * rp.im;   // Im(rs conj(rp))
  return m;
}

// Smooth dielectric interface (Eq. K_reflection_refraction with refraction),
// met at cos_i from the medium of index eta_a, relative index n_rel =
// eta_b / eta_a.  Reflection is chosen when u < R, the unpolarised
// reflectance (R = 1 past the critical angle), else refraction.  Returns the
// Mueller entries (as fresnel_conductor) of the chosen lobe divided by its
// probability; a refraction also carries the radiance factor (eta_a/eta_b)^2
// and the power factor n_rel cos_t / cos_i of the Born & Wolf amplitudes
// t_s = 2 cos_i / (cos_i + n_rel cos_t), t_p = 2 cos_i / (n_rel cos_i + cos_t).
__device__ __forceinline__ FresnelM dielectric_pick(float cos_i, float n_rel, float u, bool& refract, float& cos_t) {
  const float sin2_t = (1.0f - cos_i * cos_i) / (n_rel * n_rel);
  FresnelM F = fresnel_conductor(cos_i, n_rel, 0.0f);
  const bool tir = sin2_t >= 1.0f;
  const float R = tir ? 1.0f : F.a;
  refract = !(u < R);
  cos_t = 0.0f;
  if (!refract) {
    const float inv = 1.0f / R;
    F.a *= inv;
    F.b *= inv;
    F.cr *= inv;
    F.ci *= inv;
    return F;
  }
  cos_t = sqrtf(1.0f - sin2_t);
  const float ts = 2.0f * cos_i / (cos_i + n_rel * cos_t);
  const float tp = 2.0f * cos_i / (n_rel * cos_i + cos_t);
  const float ratio = 1.0f / n_rel;  // eta_a / eta_b
  const float f = (n_rel * cos_t / cos_i) * (ratio * ratio) / (1.0f - R);
  F.a = 0.5f * (ts * ts + tp * tp) * f;
  F.b = 0.5f * (ts * ts - tp * tp) * f;
  F.cr = ts * tp * f;
  F.ci = 0.0f;
  return F;
}

// s vector of the plane of incidence for propagation k at normal n; falls back
// to `fb` (orthogonalised against k) near normal incidence.
__device__ __forceinline__ float3 s_vector(float3 n, float3 k, float3 fb) {
  float3 s = cross(n, k);
  float l2 = dot(s, s);
  if (l2 > 1e-14f) return rsqrtf(l2) * s;
  return normalize(fb - dot(fb, k) * k);
}

}  // namespace gr
