// FP64 CPU oracle for backward Monte Carlo path tracing of generalized rays.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
// calls this file; only tests/, __graft_entry__.smoke() and bench.py's
// cpu_baseline / reference arm use it (through oracle/oracle.py).  It shares no
// header, helper, constant table or generator with the CUDA path: the two agree
// only on the plain input arrays written by the seeded scene generator and on
// the published definitions both follow (Philox4x32-10, the duff ONB, the
// paper's equations).
//
// Everything here is plain, slow, double precision, written step by step in the
// order of the paper's rendering algorithm (Algorithm 1, with the interactive
// simplifications of Sec. 7.2):
//   source a generalized ray from the pixel          (Eq. MC_sourcing)
//   propagate it (closest hit, footprint update)     (Eq. K_free_space_propagation)
//   measure it against light sources                 (Eq. measurement_operator)
//   interact with the wavevector reversed            (Eq. action_time_reversal)
//     grating orders                                 (Eq. K_grating)
//     rough-surface lobe                             (Eq. K_surface_HS)
//     smooth reflection with Fresnel weight          (Eq. K_reflection_refraction)
//   sample the scattered distribution, update weight (Eq. MC_light_transport_Q1)
// plus next-event estimation and Russian roulette (Sec. 7.2, implementation
// details).  Where the paper leaves a quantity open, the reading used is stated
// in the comment at that line; the same list of readings is kept with the
// project's design notes.
//
// Units: scene geometry in metres; optical lengths (wavelength, grating period
// and height, roughness, correlation and coherence lengths, beta) in
// micrometres.  |k| = 2*pi/lambda in 1/um (refractive index 1, Sec. 3.1).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

const double PI = 3.14159265358979323846;

// ---------------------------------------------------------------- vectors
struct V3 {
  double x, y, z;
};
V3 v3(double x, double y, double z) { return V3{x, y, z}; }
V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
V3 neg(V3 a) { return v3(-a.x, -a.y, -a.z); }
double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
V3 cross(V3 a, V3 b) {
  return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
double length(V3 a) { return std::sqrt(dot(a, a)); }
V3 normalize(V3 a) { return (1.0 / length(a)) * a; }

// Orthonormal basis around a unit vector n: the branchless construction of
// Duff, Burgess, Christensen, Hery, Kensler, Liani, Villemin, "Building an
// Orthonormal Basis, Revisited", JCGT 6(1), 2017.  The choice of basis fixes
// how the two Gaussian random numbers of a transverse sample map to space.
void onb(V3 n, V3* e1, V3* e2) {
  double sign = std::copysign(1.0, n.z);
  double a = -1.0 / (sign + n.z);
  double b = n.x * n.y * a;
  *e1 = v3(1.0 + sign * n.x * n.x * a, sign * b, -sign * n.x);
  *e2 = v3(b, sign + n.y * n.y * a, -n.y);
}

// ---------------------------------------------------------------- RNG
// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11): ten rounds of the
// 4x32 Philox S-box, multipliers 0xD2511F53 / 0xCD9E8D57, Weyl key bumps
// 0x9E3779B9 / 0xBB67AE85, the key bumped before every round but the first.
void philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0;
    c1 = n1;
    c2 = n2;
    c3 = n3;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

// Random-number addressing (fixed convention of this project, both sides):
//   key     = (seed, view index)
//   counter = (pixel index y*W+x, sample index, (segment << 4) | call, 0)
// segment = number of surface interactions before the current ray segment
// (0 for the camera ray); the call identifies the use at the vertex that ends
// that segment.  Each 32-bit word maps to u = (x >> 8) * 2^-24 in [0,1), which
// is exact in both float and double.
enum Call { CALL_JITTER = 0, CALL_EMIT_FOOT = 1, CALL_LOBE = 2, CALL_NEE_DIR = 3, CALL_NEE_FOOT = 4, CALL_RR = 5 };

struct Rng {
  uint32_t key[2];
  uint32_t pixel;
  uint32_t sample;
  void draw(int segment, int call, double u[4]) const {
    uint32_t ctr[4] = {pixel, sample, ((uint32_t)segment << 4) | (uint32_t)call, 0u};
    uint32_t x[4];
    philox4x32_10(ctr, key, x);
    for (int i = 0; i < 4; ++i) u[i] = (double)(x[i] >> 8) * (1.0 / 16777216.0);
  }
};

// Two independent standard normals from two uniforms (Box & Muller 1958).
// 1-u is used so the logarithm's argument lies in (0, 1].
void box_muller(double u0, double u1, double* z0, double* z1) {
  double r = std::sqrt(-2.0 * std::log(1.0 - u0));
  double phi = 2.0 * PI * u1;
  *z0 = r * std::cos(phi);
  *z1 = r * std::sin(phi);
}

// ---------------------------------------------------------------- special functions
// Bessel function of the first kind of integer order, by its power series
// J_n(x) = sum_m (-1)^m (x/2)^(2m+n) / (m! (m+n)!)   (A&S 9.1.10).
double bessel_j(int n, double x) {
  double sgn = 1.0;
  if (n < 0) {
    n = -n;
    if (n & 1) sgn = -1.0;  // J_{-n} = (-1)^n J_n
  }
  double half = 0.5 * x;
  double term = 1.0;
  for (int i = 1; i <= n; ++i) term *= half / i;  // (x/2)^n / n!
  double sum = term;
  for (int m = 1; m < 200; ++m) {
    term *= -(half * half) / ((double)m * (double)(m + n));
    sum += term;
    if (std::fabs(term) < 1e-18 * std::fabs(sum) && m > 2) break;
  }
  return sgn * sum;
}

// von Mises-Fisher density on the unit sphere about mean direction mu with
// concentration kappa (reading of the angular Gaussian measurement lobe on the
// sphere): kappa / (2 pi (1 - e^{-2 kappa})) * exp(-kappa |w - mu|^2 / 2).
double vmf(V3 w, V3 mu, double kappa) {
  if (kappa < 1e-8) return 1.0 / (4.0 * PI);
  V3 d = w - mu;
  return kappa / (2.0 * PI * (-std::expm1(-2.0 * kappa))) * std::exp(-0.5 * kappa * dot(d, d));
}

// Sample a direction from the vMF about mu (Wood 1994 / Jakob 2012 form):
// 1 - cos(theta) = -log(u' + (1-u') e^{-2 kappa}) / kappa with u' = 1-u0.
V3 vmf_sample(V3 mu, double kappa, double u0, double u1) {
  double up = 1.0 - u0;
  double v = -std::log(up + (1.0 - up) * std::exp(-2.0 * kappa)) / kappa;  // 1 - cos
  double sin_t = std::sqrt(std::max(0.0, v * (2.0 - v)));
  double phi = 2.0 * PI * u1;
  V3 e1, e2;
  onb(mu, &e1, &e2);
  return normalize((sin_t * std::cos(phi)) * e1 + (sin_t * std::sin(phi)) * e2 + (1.0 - v) * mu);
}

// ---------------------------------------------------------------- scene
enum MatType { MAT_ABSORBER = 0, MAT_GRATING = 1, MAT_ROUGH = 2, MAT_MIRROR = 3, MAT_EMITTER = 4, MAT_DIELECTRIC = 5 };

struct Material {
  int type;
  int fresnel;  // 0: unit reflectance (Mueller identity), 1: conductor (n + i kappa)
  double n_re, n_im;
  double period_um, height_um;
  V3 gdir;
  double sigma_h_um, corr_len_um;
  double Le, coh_len_um;
  double cauchy_b_um2;  // dielectric: index n(lambda) = n_re + cauchy_b_um2 / lambda^2
};

struct Light {
  int type;  // 0: distant source, 1: constant environment
  V3 dir;    // unit vector toward the source
  double E;
  double coh_len_um;
};

struct Tri {
  V3 v0, v1, v2;
  int mat;
};

struct Box {
  V3 lo, hi;
};

struct BvhNode {
  Box box;
  int left, right;  // children (internal) or -1
  int first, count; // triangle range in order[] (leaf)
};

struct Scene {
  std::vector<Tri> tris;
  std::vector<Material> mats;
  std::vector<Light> lights;
  // Emitters: an emitter is the planar set of triangles that share one emitter
  // material (a quad is two triangles); emitters[i] lists triangle ids and
  // emitter_of_mat maps a material id to its emitter index (or -1).
  std::vector<std::vector<int>> emitters;
  std::vector<int> emitter_of_mat;
  std::vector<BvhNode> nodes;
  std::vector<int> order;
};

Box tri_box(const Tri& t) {
  Box b;
  b.lo = v3(std::min({t.v0.x, t.v1.x, t.v2.x}), std::min({t.v0.y, t.v1.y, t.v2.y}),
            std::min({t.v0.z, t.v1.z, t.v2.z}));
  b.hi = v3(std::max({t.v0.x, t.v1.x, t.v2.x}), std::max({t.v0.y, t.v1.y, t.v2.y}),
            std::max({t.v0.z, t.v1.z, t.v2.z}));
  return b;
}

// Binary bounding-volume hierarchy built top-down by the surface area
// heuristic (MacDonald & Booth 1990) over 16 centroid bins per axis, one
// triangle per leaf.  It is only an accelerator for the oracle's closest-hit
// query (checked against an exhaustive scan by the tests) and the reference
// tree whose node visits and triangle tests per query define the traversal
// work the benchmark reports, independently of the GPU's tree.
double box_half_area(const Box& b) {
  V3 e = b.hi - b.lo;
  return e.x * e.y + e.y * e.z + e.z * e.x;
}

Box box_union(const Box& a, const Box& b) {
  Box r;
  r.lo = v3(std::min(a.lo.x, b.lo.x), std::min(a.lo.y, b.lo.y), std::min(a.lo.z, b.lo.z));
  r.hi = v3(std::max(a.hi.x, b.hi.x), std::max(a.hi.y, b.hi.y), std::max(a.hi.z, b.hi.z));
  return r;
}

int build_bvh(Scene& S, int first, int count) {
  Box b = tri_box(S.tris[S.order[first]]);
  for (int i = first + 1; i < first + count; ++i) b = box_union(b, tri_box(S.tris[S.order[i]]));
  BvhNode node;
  node.box = b;
  node.left = node.right = -1;
  node.first = first;
  node.count = count;
  const int idx = (int)S.nodes.size();
  S.nodes.push_back(node);
  if (count <= 1) return idx;
  auto centroid = [&](int t) {
    const Tri& tr = S.tris[t];
    return (1.0 / 3.0) * (tr.v0 + tr.v1 + tr.v2);
  };
  auto comp = [](V3 v, int a) { return a == 0 ? v.x : (a == 1 ? v.y : v.z); };
  V3 clo = centroid(S.order[first]), chi = clo;
  for (int i = first; i < first + count; ++i) {
    V3 c = centroid(S.order[i]);
    clo = v3(std::min(clo.x, c.x), std::min(clo.y, c.y), std::min(clo.z, c.z));
    chi = v3(std::max(chi.x, c.x), std::max(chi.y, c.y), std::max(chi.z, c.z));
  }
  // best (axis, bin boundary) by SAH cost A_left n_left + A_right n_right
  const int NB = 16;
  int best_axis = -1, best_split = -1;
  double best_cost = 1e300;
  for (int a = 0; a < 3; ++a) {
    const double lo = comp(clo, a), ext = comp(chi, a) - lo;
    if (!(ext > 0.0)) continue;
    int cnt[NB] = {0};
    Box bb[NB];
    bool has[NB] = {false};
    for (int i = first; i < first + count; ++i) {
      int k = (int)(NB * (comp(centroid(S.order[i]), a) - lo) / ext);
      k = std::min(NB - 1, std::max(0, k));
      const Box t = tri_box(S.tris[S.order[i]]);
      bb[k] = has[k] ? box_union(bb[k], t) : t;
      has[k] = true;
      ++cnt[k];
    }
    // suffix areas, then sweep the boundaries left to right
    double right_area[NB];
    int right_cnt[NB];
    Box acc;
    bool any = false;
    int c = 0;
    for (int k = NB - 1; k >= 1; --k) {
      if (has[k]) {
        acc = any ? box_union(acc, bb[k]) : bb[k];
        any = true;
      }
      c += cnt[k];
      right_area[k] = any ? box_half_area(acc) : 0.0;
      right_cnt[k] = c;
    }
    any = false;
    c = 0;
    for (int k = 0; k < NB - 1; ++k) {
      if (has[k]) {
        acc = any ? box_union(acc, bb[k]) : bb[k];
        any = true;
      }
      c += cnt[k];
      if (c == 0 || right_cnt[k + 1] == 0) continue;
      const double cost = box_half_area(acc) * c + right_area[k + 1] * right_cnt[k + 1];
      if (cost < best_cost) {
        best_cost = cost;
        best_axis = a;
        best_split = k + 1;
      }
    }
  }
  int mid;
  if (best_axis < 0) {
    mid = first + count / 2;  // coincident centroids: split the range in half
  } else {
    const double lo = comp(clo, best_axis), ext = comp(chi, best_axis) - lo;
    auto left_of = [&](int t) {
      int k = (int)(NB * (comp(centroid(t), best_axis) - lo) / ext);
      k = std::min(NB - 1, std::max(0, k));
      return k < best_split;
    };
    mid = (int)(std::stable_partition(S.order.begin() + first, S.order.begin() + first + count, left_of) -
                S.order.begin());
    if (mid == first || mid == first + count) mid = first + count / 2;
  }
  const int l = build_bvh(S, first, mid - first);
  const int r = build_bvh(S, mid, first + count - mid);
  S.nodes[idx].left = l;
  S.nodes[idx].right = r;
  S.nodes[idx].count = 0;
  return idx;
}

// Ray-triangle intersection (Moller & Trumbore 1997), double precision, edges
// inclusive.  Returns the distance t or -1.
double intersect_tri(const Tri& T, V3 o, V3 d) {
  V3 e1 = T.v1 - T.v0, e2 = T.v2 - T.v0;
  V3 p = cross(d, e2);
  double det = dot(e1, p);
  if (det == 0.0) return -1.0;
  double inv = 1.0 / det;
  V3 s = o - T.v0;
  double u = dot(s, p) * inv;
  if (u < 0.0 || u > 1.0) return -1.0;
  V3 q = cross(s, e1);
  double v = dot(d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return -1.0;
  return dot(e2, q) * inv;
}

// Self-intersection guard shared by the convention of both implementations:
// hits closer than T_MIN metres, and the primitive just left, are ignored.
const double T_MIN = 1e-5;

// Entry distance of the ray into the box (>= 0), or -1 when it misses the box
// or enters beyond tmax.
double box_entry(const Box& b, V3 o, V3 d, double tmax) {
  double t0 = 0.0, t1 = tmax;
  double oo[3] = {o.x, o.y, o.z}, dd[3] = {d.x, d.y, d.z};
  double lo[3] = {b.lo.x, b.lo.y, b.lo.z}, hi[3] = {b.hi.x, b.hi.y, b.hi.z};
  for (int a = 0; a < 3; ++a) {
    if (dd[a] == 0.0) {
      if (oo[a] < lo[a] || oo[a] > hi[a]) return -1.0;
      continue;
    }
    double ta = (lo[a] - oo[a]) / dd[a], tb = (hi[a] - oo[a]) / dd[a];
    if (ta > tb) std::swap(ta, tb);
    // widen by a relative margin so the box test never rejects a triangle hit
    double pad = 1e-9 * (std::fabs(ta) + std::fabs(tb)) + 1e-12;
    ta -= pad;
    tb += pad;
    t0 = std::max(t0, ta);
    t1 = std::min(t1, tb);
    if (t0 > t1) return -1.0;
  }
  return t0;
}

// Traversal work of the closest-hit queries made since the last reset, over
// every thread: queries, internal node visits (two child boxes tested each)
// and ray-triangle tests.
std::atomic<long long> g_work_queries{0}, g_work_visits{0}, g_work_tests{0};

// Closest hit with t > T_MIN, excluding one primitive; equal distances resolve
// to the lower primitive id.
bool closest_hit(const Scene& S, V3 o, V3 d, int exclude, bool use_bvh, double* t_out, int* prim_out) {
  double best = 1e300;
  int bi = -1;
  long long visits = 0, tests = 0;
  auto test = [&](int i) {
    if (i == exclude) return;
    ++tests;
    double t = intersect_tri(S.tris[i], o, d);
    if (t > T_MIN && (t < best || (t == best && i < bi))) {
      best = t;
      bi = i;
    }
  };
  if (!use_bvh || S.nodes.empty()) {
    for (int i = 0; i < (int)S.tris.size(); ++i) test(i);
  } else if (S.nodes[0].left < 0) {
    test(S.order[S.nodes[0].first]);
  } else {
    // nearer child first, the farther one stacked; leaf children tested at once
    std::vector<int> stack;
    int ni = 0;
    for (;;) {
      ++visits;
      const BvhNode& n = S.nodes[ni];
      int next[2];
      double tn[2];
      int m = 0;
      for (int c = 0; c < 2; ++c) {
        const int ch = c == 0 ? n.left : n.right;
        const BvhNode& cn = S.nodes[ch];
        const double te = box_entry(cn.box, o, d, best);
        if (te < 0.0) continue;
        if (cn.left < 0) {
          test(S.order[cn.first]);
        } else {
          next[m] = ch;
          tn[m] = te;
          ++m;
        }
      }
      if (m == 2) {
        const bool swap = tn[1] < tn[0];
        stack.push_back(swap ? next[0] : next[1]);
        ni = swap ? next[1] : next[0];
        continue;
      }
      if (m == 1) {
        ni = next[0];
        continue;
      }
      // pop, skipping subtrees now beyond the best hit
      ni = -1;
      while (!stack.empty()) {
        const int cand = stack.back();
        stack.pop_back();
        if (box_entry(S.nodes[cand].box, o, d, best) >= 0.0) {
          ni = cand;
          break;
        }
      }
      if (ni < 0) break;
    }
  }
  g_work_queries.fetch_add(1, std::memory_order_relaxed);
  g_work_visits.fetch_add(visits, std::memory_order_relaxed);
  g_work_tests.fetch_add(tests, std::memory_order_relaxed);
  if (bi < 0) return false;
  *t_out = best;
  *prim_out = bi;
  return true;
}

V3 tri_normal(const Tri& T) { return normalize(cross(T.v1 - T.v0, T.v2 - T.v0)); }

// ---------------------------------------------------------------- view
struct View {
  V3 eye, look, up;
  double vfov_deg;
  int W, H;
  double p_pix_um, f_beta;
  double lmin_um, lmax_um;
  int n_bins, n_stokes, max_depth;
  long spp, first_sample;
  uint32_t view_index;
  int ortho;
  double ortho_half_m;
};

// Wavelength of bin b: lambda_b = lambda_min + b (lambda_max - lambda_min)/(n_bins - 1)
// (reading of the hero wavelength as one discrete bin per path, stratified by
// sample index: b = s mod n_bins).
double bin_lambda(const View& V, int b) {
  if (V.n_bins <= 1) return V.lmin_um;
  return V.lmin_um + (double)b * (V.lmax_um - V.lmin_um) / (double)(V.n_bins - 1);
}

// Number of the view's samples s in [first_sample, first_sample + spp) whose
// bin s mod n_bins is b.
long bin_count(const View& V, int b) {
  long n = 0;
  for (long s = V.first_sample; s < V.first_sample + V.spp; ++s) n += (s % V.n_bins) == b;
  return n;
}

// ---------------------------------------------------------------- free-space propagation
// Eq. K_free_space_propagation with zbar = z/|k0| (z in um):
//   beta_o^2 = beta^2 + 2 zbar rho + zbar^2 (1 + rho^2) / beta^2
//   rho_o    = rho + zbar (1 + rho^2) / beta^2
void propagate(double* beta2, double* rho, double zbar) {
  double b2 = *beta2, r = *rho;
  double b2o = b2 + 2.0 * zbar * r + zbar * zbar * (1.0 + r * r) / b2;
  double ro = r + zbar * (1.0 + r * r) / b2;
  *beta2 = b2o;
  *rho = ro;
}

// ---------------------------------------------------------------- polarisation
typedef std::complex<double> cplx;

// Fresnel amplitude reflection coefficients of a smooth conductor with
// complex index n = n_re + i n_im (Born & Wolf, Sec. 1.5 / 14.2 sign choice, so
// that r_p = -r_s at normal incidence):
//   r_s = (cos_i - n cos_t) / (cos_i + n cos_t),  r_p = (n cos_i - cos_t) / (n cos_i + cos_t)
// with n cos_t = sqrt(n^2 - sin_i^2) (principal branch).
void fresnel_conductor(double cos_i, double n_re, double n_im, cplx* rs, cplx* rp) {
  cplx n(n_re, n_im);
  double sin2 = std::max(0.0, 1.0 - cos_i * cos_i);
  cplx n_cos_t = std::sqrt(n * n - sin2);
  cplx cos_t = n_cos_t / n;
  *rs = (cos_i - n_cos_t) / (cos_i + n_cos_t);
  *rp = (n * cos_i - cos_t) / (n * cos_i + cos_t);
}

struct M4 {
  double m[4][4];
};
M4 m4_identity() {
  M4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) r.m[i][j] = (i == j) ? 1.0 : 0.0;
  return r;
}
M4 m4_mul(const M4& a, const M4& b) {
  M4 r;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += a.m[i][k] * b.m[k][j];
      r.m[i][j] = s;
    }
  return r;
}

// Mueller matrix of the Jones matrix diag(a, b) in an (s, p) basis, Stokes
// convention S = (|Es|^2+|Ep|^2, |Es|^2-|Ep|^2, 2 Re(Es Ep*), -2 Im(Es Ep*)).
M4 mueller_diag(cplx a, cplx b) {
  double A = std::norm(a), B = std::norm(b);
  cplx c = a * std::conj(b);
  M4 r;
  std::memset(&r, 0, sizeof r);
  r.m[0][0] = 0.5 * (A + B);
  r.m[0][1] = 0.5 * (A - B);
  r.m[1][0] = 0.5 * (A - B);
  r.m[1][1] = 0.5 * (A + B);
  r.m[2][2] = c.real();
  r.m[2][3] = c.imag();
  r.m[3][2] = -c.imag();
  r.m[3][3] = c.real();
  return r;
}

// Smooth dielectric interface (Eq. K_reflection_refraction, with refraction):
// light meets the interface from the medium of index eta_a at cos_i, the far
// side has eta_b; n_rel = eta_b / eta_a.  Born & Wolf amplitudes with
// cos_t = sqrt(1 - (1 - cos_i^2) / n_rel^2):
//   r_s = (cos_i - n_rel cos_t) / (cos_i + n_rel cos_t)
//   r_p = (n_rel cos_i - cos_t) / (n_rel cos_i + cos_t)
//   t_s = 2 cos_i / (cos_i + n_rel cos_t),  t_p = 2 cos_i / (n_rel cos_i + cos_t)
// and power transmittances T_x = (n_rel cos_t / cos_i) |t_x|^2, so that
// R_x + T_x = 1.  Past the critical angle cos_t is imaginary, |r_s| = |r_p| = 1
// and nothing is transmitted.  R, T are the unpolarised averages.
struct Dielectric {
  cplx rs, rp;
  double ts, tp;
  double cos_t;
  bool tir;
  double R, T;
};
void fresnel_dielectric(double cos_i, double n_rel, Dielectric* D) {
  fresnel_conductor(cos_i, n_rel, 0.0, &D->rs, &D->rp);
  const double sin2_t = (1.0 - cos_i * cos_i) / (n_rel * n_rel);
  D->tir = sin2_t >= 1.0;
  if (D->tir) {
    D->cos_t = 0.0;
    D->ts = D->tp = 0.0;
    D->R = 1.0;
    D->T = 0.0;
    return;
  }
  D->cos_t = std::sqrt(1.0 - sin2_t);
  D->ts = 2.0 * cos_i / (cos_i + n_rel * D->cos_t);
  D->tp = 2.0 * cos_i / (n_rel * cos_i + D->cos_t);
  D->R = 0.5 * (std::norm(D->rs) + std::norm(D->rp));
  const double f = n_rel * D->cos_t / cos_i;
  D->T = 0.5 * f * (D->ts * D->ts + D->tp * D->tp);
}

// Refracted unit direction (Snell's law in vector form) for incidence d on a
// surface whose normal n faces the incident side (dot(d, n) < 0).
V3 refract_dir(V3 d, V3 n, double n_rel, double cos_i, double cos_t) {
  const double e = 1.0 / n_rel;
  return e * d + (e * cos_i - cos_t) * n;
}

// Rotation of the Stokes reference frame: frame B's x axis at angle phi from
// frame A's x axis (counter-clockwise about the common propagation direction).
M4 stokes_rotation(double phi) {
  M4 r = m4_identity();
  double c = std::cos(2.0 * phi), s = std::sin(2.0 * phi);
  r.m[1][1] = c;
  r.m[1][2] = s;
  r.m[2][1] = -s;
  r.m[2][2] = c;
  return r;
}

// Angle of frame B's x axis measured in frame A = (xa, ya).
double frame_angle(V3 xa, V3 ya, V3 xb) { return std::atan2(dot(xb, ya), dot(xb, xa)); }

// s vector of a plane of incidence for light propagating along k at a surface
// with normal n: normalize(n x k); near normal incidence it is undefined and the
// fallback vector (orthogonalised against k) is used instead.
V3 s_vector(V3 n, V3 k, V3 fallback) {
  V3 s = cross(n, k);
  double l = length(s);
  if (l > 1e-7) return (1.0 / l) * s;
  V3 f = fallback - dot(fallback, k) * k;
  return normalize(f);
}

// ---------------------------------------------------------------- path state
struct PathState {
  V3 o, d;         // mean position (m) and unit propagation direction of the ray
  double beta2;    // beta^2 (um^2)
  double rho;
  double k;        // |k0| (1/um)
  double lambda;   // um
  double eta;      // refractive index of the medium the ray travels in (1 = air)
  double s_ray2;   // invariant angular variance (sigma_k/|k|)^2 (rad^2)
  int prev_prim;
  // throughput: scalar (n_stokes == 1) or Mueller matrix with frame x axis
  double t;
  M4 T;
  V3 xf;
  // MIS bookkeeping for the vertex that produced the current segment
  bool prev_delta;  // true after the camera, a specular lobe, a grating order or a mirror
  double prev_pdf;  // solid-angle density of the current direction at that vertex
  // anisotropic footprint (FLAG_ANISO): K = A^{-1} (um^2) of the transverse
  // field exp(-x^T A x / 2), x in the frame (xf, d x xf); entries K11, K12, K22
  cplx K[3];
};

struct Ctx {
  const Scene* S;
  const View* V;
  int flags;
  Rng rng;
};
const int FLAG_NEE = 1, FLAG_RR = 2, FLAG_NO_RENORM = 4, FLAG_HERO = 16, FLAG_ANISO = 32;

// Angular spread of a source of coherence length lc (Eq. coherence_diffusivity
// read per axis with Theta = lc^2): s_src = lambda / lc; lc = 0 means spatially
// coherent (s_src = 0).
double source_spread2(double lambda, double lc) {
  if (lc <= 0.0) return 0.0;
  double s = lambda / lc;
  return s * s;
}

// Measurement operator (Eq. measurement_operator) for a distant source: the
// k-marginal of the generalized ray (Gaussian of angular variance s_ray^2)
// convolved with the source's angular spread, evaluated on the sphere as a vMF
// of concentration 1/(s_ray^2 + s_src^2) about the source direction.
double measure_distant(const Light& L, V3 d, double lambda, double s_ray2) {
  if (L.type == 1) return L.E;  // constant environment
  double kappa = 1.0 / (s_ray2 + source_spread2(lambda, L.coh_len_um));
  return L.E * vmf(d, L.dir, kappa);
}

// Coverage of the footprint point p (m), projected along d onto the plane of
// emitter triangle prim: inside any triangle of the emitter (barycentric test,
// edges inclusive); the emitter's triangles are coplanar.
bool emitter_covers(const Scene& S, int prim, V3 p, V3 d) {
  const Tri& T = S.tris[prim];
  V3 ne = tri_normal(T);
  double tp = dot(T.v0 - p, ne) / dot(d, ne);
  V3 q = p + tp * d;
  for (int ti : S.emitters[S.emitter_of_mat[T.mat]]) {
    const Tri& E = S.tris[ti];
    V3 a = E.v1 - E.v0, b = E.v2 - E.v0, c = q - E.v0;
    double daa = dot(a, a), dab = dot(a, b), dbb = dot(b, b), dca = dot(c, a), dcb = dot(c, b);
    double den = daa * dbb - dab * dab;
    double bu = (dbb * dca - dab * dcb) / den;
    double bv = (daa * dcb - dab * dca) / den;
    if (bu >= 0.0 && bv >= 0.0 && bu + bv <= 1.0) return true;
  }
  return false;
}

// Measurement operator for an emissive triangle hit by the ray (Eq.
// measurement_operator restricted to the source's support, Sec. 7.2 emissive
// geometry): one transverse point x ~ N(0, beta^2/2) of the footprint is drawn,
// projected along d onto the emitter plane and tested for coverage; the local
// mean direction there is shifted by rho x / (beta^2 |k|) (the conditional
// mean of the phase-space Gaussian given position) with residual angular
// variance 1/(2 beta^2 |k|^2); the source emits a Gaussian lobe of spread
// s_src about its normal.
double measure_emitter(const Scene& S, int prim, V3 hit, V3 d, double beta2, double rho, double k, double lambda,
                       double ua, double ub) {
  const Tri& T = S.tris[prim];
  const Material& M = S.mats[T.mat];
  V3 ne = tri_normal(T);
  if (dot(d, ne) >= 0.0) return 0.0;  // one-sided: only the front face emits
  double z0, z1;
  box_muller(ua, ub, &z0, &z1);
  double sigma = std::sqrt(0.5 * beta2);  // um
  V3 e1, e2;
  onb(d, &e1, &e2);
  V3 x_um = (sigma * z0) * e1 + (sigma * z1) * e2;
  if (!emitter_covers(S, prim, hit + 1e-6 * x_um, d)) return 0.0;
  V3 mu = (rho / (beta2 * k)) * x_um;
  V3 dl = normalize(d + mu);
  double sc2 = 1.0 / (2.0 * beta2 * k * k);
  double kappa = 1.0 / (sc2 + source_spread2(lambda, M.coh_len_um));
  return M.Le * vmf(neg(dl), ne, kappa);
}

// ---------------------------------------------------------------- anisotropic footprints
// Anisotropic generalized rays (beta and rho as matrices; Sec. 3.1 and the
// definition of the generalized ray, Eq. def_gen_ray, leave the general form
// to a supplemental that is not available; this is our derivation).  The
// transverse field of a generalized ray is exp(-x^T A x / 2) with A complex
// symmetric and Re A positive definite; the scalar ray is A = (1 - i rho) /
// beta^2.  The state kept is K = A^{-1}:
//  - free-space propagation (the paraxial transfer function exp(-i zbar
//    |k_t|^2 / 2), zbar = z/|k|) gives K <- K + i zbar I, which for the
//    scalar ray is Eq. K_free_space_propagation;
//  - the wavevector marginal is Gaussian with covariance Re(K)^{-1} / 2, the
//    spatial marginal has covariance Re(A)^{-1} / 2, and given position x the
//    wavevector has mean -Im(A) x and covariance Re(A) / 2 (the Wigner
//    function of the Gaussian field);
//  - an interaction with a surface matches the field on the surface: with
//    P_in, P_out the projections of a tangent basis onto the incident and
//    outgoing transverse frames, K_out = W K W^T, W = P_out P_in^{-1} (the
//    anamorphic map; orthogonal for mirror reflection).
struct CS2 {
  cplx a, b, c;  // [[a, b], [b, c]]
};

CS2 cs2_inverse(const CS2& K) {
  const cplx det = K.a * K.c - K.b * K.b;
  return CS2{K.c / det, -K.b / det, K.a / det};
}

// W K W^T for a real 2x2 W
CS2 cs2_congruence(const double W[2][2], const CS2& K) {
  CS2 r;
  r.a = W[0][0] * W[0][0] * K.a + 2.0 * W[0][0] * W[0][1] * K.b + W[0][1] * W[0][1] * K.c;
  r.b = W[0][0] * W[1][0] * K.a + (W[0][0] * W[1][1] + W[0][1] * W[1][0]) * K.b + W[0][1] * W[1][1] * K.c;
  r.c = W[1][0] * W[1][0] * K.a + 2.0 * W[1][0] * W[1][1] * K.b + W[1][1] * W[1][1] * K.c;
  return r;
}

void inv2(const double M[2][2], double R[2][2]) {
  const double det = M[0][0] * M[1][1] - M[0][1] * M[1][0];
  R[0][0] = M[1][1] / det;
  R[0][1] = -M[0][1] / det;
  R[1][0] = -M[1][0] / det;
  R[1][1] = M[0][0] / det;
}

// K after an interaction at a surface of normal n: incident direction d_in
// with frame x axis f_in, outgoing direction d_out with frame x axis f_out
// (frames (f, d x f)).
CS2 aniso_interaction(const CS2& K, V3 f_in, V3 d_in, V3 f_out, V3 d_out, V3 n) {
  V3 s1, s2;
  onb(n, &s1, &s2);
  const V3 u[2] = {f_in, cross(d_in, f_in)}, v[2] = {f_out, cross(d_out, f_out)};
  double Pin[2][2], Pout[2][2], Iin[2][2], W[2][2];
  for (int i = 0; i < 2; ++i) {
    Pin[i][0] = dot(u[i], s1);
    Pin[i][1] = dot(u[i], s2);
    Pout[i][0] = dot(v[i], s1);
    Pout[i][1] = dot(v[i], s2);
  }
  inv2(Pin, Iin);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) W[i][j] = Pout[i][0] * Iin[0][j] + Pout[i][1] * Iin[1][j];
  return cs2_congruence(W, K);
}

void aniso_propagate(CS2* K, double zbar) {
  K->a += cplx(0.0, zbar);
  K->c += cplx(0.0, zbar);
}

// An angular Gaussian lobe about mu with (2D) precision matrix Ci in the
// frame (f1, f2) transverse to the lobe, written so that an isotropic Ci =
// kappa I gives the vMF of Eq. measurement_operator exactly: with kbar =
// tr(Ci) / 2 and dv = w - mu, exponent kbar |dv|^2 / 2 plus the traceless
// part (Ci - kbar I) on the transverse components of dv; normalised with the
// vMF constant of kappa_eff = sqrt(det Ci).
double aniso_lobe(V3 w, V3 mu, V3 f1, V3 f2, const double Ci[2][2]) {
  const double ke = std::sqrt(std::max(0.0, Ci[0][0] * Ci[1][1] - Ci[0][1] * Ci[1][0]));
  if (ke < 1e-8) return 1.0 / (4.0 * PI);
  const double kbar = 0.5 * (Ci[0][0] + Ci[1][1]);
  const V3 dv = w - mu;
  const double t1 = dot(dv, f1), t2 = dot(dv, f2);
  const double q = 0.5 * (kbar * dot(dv, dv) + (Ci[0][0] - kbar) * t1 * t1 + 2.0 * Ci[0][1] * t1 * t2 +
                          (Ci[1][1] - kbar) * t2 * t2);
  return ke / (2.0 * PI * (-std::expm1(-2.0 * ke))) * std::exp(-q);
}

// Distant source measured by an anisotropic ray: the wavevector marginal
// (covariance Re(K)^{-1} / 2 in k units, / |k|^2 in direction units) plus
// the source's spread.
double measure_distant_aniso(const Light& L, V3 d, double lambda, double k, const CS2& K, V3 xf) {
  if (L.type == 1) return L.E;
  const double ReK[2][2] = {{K.a.real(), K.b.real()}, {K.b.real(), K.c.real()}};
  double C[2][2], Ci[2][2];
  inv2(ReK, C);
  const double s2 = source_spread2(lambda, L.coh_len_um);
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) C[i][j] = 0.5 * C[i][j] / (k * k) + (i == j ? s2 : 0.0);
  inv2(C, Ci);
  return L.E * aniso_lobe(d, L.dir, xf, cross(d, xf), Ci);
}

// Emitter measured by an anisotropic ray: the footprint point is drawn from
// the spatial marginal (Cholesky factor in the frame onb(d), so that an
// isotropic footprint draws the same point as measure_emitter), its direction
// shifted by -Im(A) x / |k|, with residual angular covariance Re(A) / (2 |k|^2)
// plus the source's spread.
struct AnisoFoot {
  V3 e1, e2;         // frame onb(d)
  double x1, x2;     // footprint point (um) in that frame
  double m1, m2;     // direction shift there
  double Ar[2][2];   // Re A in that frame
};

// The footprint point for the standard normal pair (z0, z1) and its
// conditional direction shift.
AnisoFoot aniso_footprint(V3 d, const CS2& K, V3 xf, double k, double z0, double z1) {
  AnisoFoot F;
  onb(d, &F.e1, &F.e2);
  const V3 u2 = cross(d, xf);
  const double R[2][2] = {{dot(F.e1, xf), dot(F.e1, u2)}, {dot(F.e2, xf), dot(F.e2, u2)}};
  const CS2 A = cs2_inverse(cs2_congruence(R, K));
  const double Ai[2][2] = {{A.a.imag(), A.b.imag()}, {A.b.imag(), A.c.imag()}};
  F.Ar[0][0] = A.a.real();
  F.Ar[0][1] = F.Ar[1][0] = A.b.real();
  F.Ar[1][1] = A.c.real();
  double Sg[2][2];
  inv2(F.Ar, Sg);
  const double l11 = std::sqrt(0.5 * Sg[0][0]), l21 = 0.5 * Sg[1][0] / l11;
  const double l22 = std::sqrt(std::max(0.0, 0.5 * Sg[1][1] - l21 * l21));
  F.x1 = l11 * z0;
  F.x2 = l21 * z0 + l22 * z1;
  F.m1 = -(Ai[0][0] * F.x1 + Ai[0][1] * F.x2) / k;
  F.m2 = -(Ai[1][0] * F.x1 + Ai[1][1] * F.x2) / k;
  return F;
}

// The emitter lobe seen from the footprint point F (covered), source spread
// s2 about the emitter normal ne, unit exitance.
double aniso_emitter_lobe(const AnisoFoot& F, V3 d, double k, double s2, V3 ne) {
  const V3 dl = normalize(d + F.m1 * F.e1 + F.m2 * F.e2);
  double C[2][2], Ci[2][2];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) C[i][j] = 0.5 * F.Ar[i][j] / (k * k) + (i == j ? s2 : 0.0);
  inv2(C, Ci);
  return aniso_lobe(neg(dl), ne, F.e1, F.e2, Ci);
}

double measure_emitter_aniso(const Scene& S, int prim, V3 hit, V3 d, const CS2& K, V3 xf, double k, double lambda,
                             double ua, double ub) {
  const Tri& T = S.tris[prim];
  const Material& M = S.mats[T.mat];
  V3 ne = tri_normal(T);
  if (dot(d, ne) >= 0.0) return 0.0;
  double z0, z1;
  box_muller(ua, ub, &z0, &z1);
  const AnisoFoot F = aniso_footprint(d, K, xf, k, z0, z1);
  if (!emitter_covers(S, prim, hit + 1e-6 * (F.x1 * F.e1 + F.x2 * F.e2), d)) return 0.0;
  return M.Le * aniso_emitter_lobe(F, d, k, source_spread2(lambda, M.coh_len_um), ne);
}

// ---------------------------------------------------------------- interactions
// Diffraction grating (Eq. K_grating): orders j with weight J_j(h k / 2)^2 and
// tangential direction cosines t_j = t_in + j (lambda/Lambda) g (the grating
// equation sin(theta_o) = sin(theta_i) - j lambda/Lambda, written in the
// conical vector form; the sign of j is immaterial as J_{-j}^2 = J_j^2).
// Evanescent orders (|t_j| >= 1) are dropped and the weights renormalised over
// the propagating ones (reading; FLAG_NO_RENORM keeps the raw weights).
struct Lobes {
  int n;
  int order[128];
  double w[128];
  V3 dir[128];
  double total;
};
void grating_lobes(const Material& M, V3 d_in, V3 n, double lambda, bool renorm, Lobes* L) {
  V3 t_in = d_in - dot(d_in, n) * n;
  V3 g = M.gdir - dot(M.gdir, n) * n;
  if (length(g) < 1e-9) {
    V3 e1, e2;
    onb(n, &e1, &e2);
    g = e1;
  }
  g = normalize(g);
  double x = PI * M.height_um / lambda;  // h k / 2
  double step = lambda / M.period_um;
  int jmax = (int)std::floor(2.0 / step) + 1;
  if (jmax > 63) jmax = 63;
  L->n = 0;
  L->total = 0.0;
  for (int j = -jmax; j <= jmax; ++j) {
    V3 t = t_in + (j * step) * g;
    double tt = dot(t, t);
    if (tt >= 1.0) continue;
    double J = bessel_j(j, x);
    int i = L->n++;
    L->order[i] = j;
    L->w[i] = J * J;
    L->dir[i] = t + std::sqrt(1.0 - tt) * n;
    L->total += J * J;
  }
  if (!renorm) L->total = 1.0;
}

// Rough surface lobe (Eq. K_surface_HS with the Harvey-Shack f_HS read as the
// Kirchhoff series of a Gaussian-correlated surface, Beckmann & Spizzichino
// 1963): roughness parameter g = (2 |k| sigma_h cos(theta_i))^2; specular part
// with weight e^{-g}; term m >= 1 (Poisson weight e^{-g} g^m / m!) is a 2D
// Gaussian in tangential direction cosines about the mirror direction with
// per-axis variance 2m / (|k| l)^2.  For g > 50 the series is replaced by its
// continuous limit, a single Gaussian with m = g and no specular part.
// Samples landing at |t| >= 1 are evanescent and carry no energy (weight 0).
const double G_CONT = 50.0;

double gauss2(V3 delta, double var) { return std::exp(-0.5 * dot(delta, delta) / var) / (2.0 * PI * var); }

// Density of the diffuse (m >= 1) part in tangential direction cosines.
double rough_diffuse_density(double g, double k, double ell, V3 delta) {
  double kl2 = (k * ell) * (k * ell);
  if (g > G_CONT) return gauss2(delta, 2.0 * g / kl2);
  double p = std::exp(-g);
  double cdf = p;
  double sum = 0.0;
  // include every m the sampler can return (until the Poisson CDF passes 1 - 2^-24)
  for (int m = 1; m < 1000; ++m) {
    p *= g / m;
    cdf += p;
    sum += p * gauss2(delta, 2.0 * m / kl2);
    if (cdf > 1.0 - 1.0 / 16777216.0 && p < 1e-12) break;
  }
  return sum;
}

// ---------------------------------------------------------------- one path sample
void add_vec(double* acc, int ns, const double* v, double s) {
  for (int i = 0; i < ns; ++i) acc[i] += v[i] * s;
}

// Throughput applied to an unpolarised source of unit intensity: first column.
void throughput_column(const PathState& P, int ns, double* out) {
  if (ns == 1) {
    out[0] = P.t;
    return;
  }
  for (int i = 0; i < 4; ++i) out[i] = P.T.m[i][0];
}

// The state one path sample carries (Algorithm 1): the generalized ray and
// its throughput, the anisotropic footprint (FLAG_ANISO, R25) and the
// hero-wavelength class (FLAG_HERO, R24), with the sample's result.
//
// Hero-wavelength spectral MIS (Sec. 7.2, after Wilkie et al. 2014): the
// path's bin is the hero of the class of G = 4 bins {c, c+Q, c+2Q, c+3Q}
// (Q = n_bins / 4) and drives every sampling decision.  q[g] is the
// probability density of the path sampled so far at class bin g's
// wavelength divided by its density at the hero's; it stays 1 through
// wavelength-independent decisions and drops to 0 at a dispersive delta
// (a grating order j != 0, a dispersive dielectric), where no other
// wavelength could have made the same path.  Every connection to a light is
// measured at each class wavelength (with that wavelength's footprint,
// carried along the path in b2/rho) and weighted by multiple importance
// sampling over the techniques that could have made the path, with
// cf_j = share of the class's samples whose hero is bin j:
//  - an escape, or an emitter hit whose last direction only the lobe could
//    have sampled: balance heuristic over the class wavelengths,
//    T M_g cf_g q_g / sum_j cf_j q_j;
//  - an emitter hit after a diffuse rough vertex, and next-event estimation,
//    with NEE on: power heuristic over the eight (wavelength j, technique t
//    = lobe or emitter sampling) pairs with full path densities
//    cf_j P_j p_{j,t}; with one hero per class it is the plain estimator's
//    power heuristic between lobe and emitter sampling.
// result[4 g + k] is class bin g's Stokes component k.
struct HeroClass {
  bool on = false;
  int G = 1, gh = 0, c0 = 0;
  double lam[4], k[4], cf[4];
  double q[4];        // path density at class wavelength g over the hero's
  double qpre[4];     // q before the latest interaction
  double b2[4], rho[4];  // the footprint the path has at class wavelength g
  void drop_companions() {
    for (int g = 0; g < G; ++g)
      if (g != gh) q[g] = 0.0;
  }
};

struct Sample {
  const Ctx& C;
  const Scene& S;
  const View& V;
  int ns;
  Rng rng;
  double* result;
  PathState P;
  bool aniso;
  CS2 K;          // anisotropic footprint (FLAG_ANISO)
  HeroClass H;
  double beta0;
  int n_emit;
  Sample(const Ctx& c, double* res)
      : C(c), S(*c.S), V(*c.V), ns(c.V->n_stokes), rng(c.rng), result(res), aniso((c.flags & FLAG_ANISO) != 0) {}
  // the vMF density of emitter sampling toward w at class wavelength g
  double nee_density(int g, V3 w, V3 ne, double coh_len_um) const {
    const double s2g = 1.0 / (2.0 * beta0 * beta0 * H.k[g] * H.k[g]);
    return vmf(w, neg(ne), 1.0 / (s2g + source_spread2(H.lam[g], coh_len_um))) / n_emit;
  }
};

// --- sourcing (Eq. MC_sourcing; Sec. 7.2): position uniform on the pixel,
// rho = 0, beta = f_beta * pixel pitch, alpha = 1, wavelength of bin s mod B.
void source(Sample& W, int px, int py, long sample) {
  const View& V = W.V;
  for (int i = 0; i < 16; ++i) W.result[i] = 0.0;
  W.rng.pixel = (uint32_t)(py * V.W + px);
  W.rng.sample = (uint32_t)sample;
  double u[4];
  W.rng.draw(0, CALL_JITTER, u);
  const int bin = (int)(sample % V.n_bins);
  PathState& P = W.P;
  P.lambda = bin_lambda(V, bin);
  P.k = 2.0 * PI / P.lambda;
  W.beta0 = V.f_beta * V.p_pix_um;
  P.beta2 = W.beta0 * W.beta0;
  P.rho = 0.0;
  P.s_ray2 = (1.0 + P.rho * P.rho) / (2.0 * P.beta2) / (P.k * P.k);
  V3 fw = normalize(V.look - V.eye);
  V3 right = normalize(cross(fw, V.up));
  V3 upc = cross(right, fw);
  double aspect = (double)V.W / (double)V.H;
  double fx = (px + u[0]) / V.W, fy = (py + u[1]) / V.H;
  if (V.ortho) {
    P.o = V.eye + ((2.0 * fx - 1.0) * V.ortho_half_m * aspect) * right + ((1.0 - 2.0 * fy) * V.ortho_half_m) * upc;
    P.d = fw;
  } else {
    double th = std::tan(0.5 * V.vfov_deg * PI / 180.0);
    double sx = (2.0 * fx - 1.0) * th * aspect;
    double sy = (1.0 - 2.0 * fy) * th;
    P.o = V.eye;
    P.d = normalize(fw + sx * right + sy * upc);
  }
  P.prev_prim = -1;
  P.eta = 1.0;
  P.t = 1.0;
  P.T = m4_identity();
  P.xf = normalize(right - dot(right, P.d) * P.d);
  P.prev_delta = true;
  P.prev_pdf = 0.0;
  W.n_emit = (int)W.S.emitters.size();
  // anisotropic footprint: the camera state is isotropic, K = beta0^2 I (rho = 0)
  W.K = CS2{cplx(P.beta2, 0.0), cplx(0.0, 0.0), cplx(P.beta2, 0.0)};
  // the hero's class: its wavelengths, sample shares and footprints
  HeroClass& H = W.H;
  H.on = (W.C.flags & FLAG_HERO) != 0;
  H.G = H.on ? 4 : 1;
  const int Qb = V.n_bins / H.G;
  H.gh = H.on ? bin / Qb : 0;
  H.c0 = bin - H.gh * Qb;
  long ncls = 0, nb_g[4];
  for (int g = 0; g < H.G; ++g) {
    H.lam[g] = bin_lambda(V, H.c0 + g * Qb);
    H.q[g] = 1.0;
    nb_g[g] = H.on ? bin_count(V, H.c0 + g * Qb) : 1;
    ncls += nb_g[g];
  }
  for (int g = 0; g < H.G; ++g) H.cf[g] = (double)nb_g[g] / (double)ncls;
  for (int g = 0; g < H.G; ++g) {
    H.qpre[g] = 1.0;
    H.b2[g] = P.beta2;
    H.rho[g] = P.rho;
    H.k[g] = 2.0 * PI / H.lam[g];
  }
}

// --- measurement of distant sources on escape (Eq. measurement_operator);
// col is the throughput column of the path
void measure_escape(Sample& W, const double* col) {
  const PathState& P = W.P;
  const HeroClass& H = W.H;
  if (!H.on) {
    double m = 0.0;
    for (const Light& L : W.S.lights)
      m += W.aniso ? measure_distant_aniso(L, P.d, P.lambda, P.k, W.K, P.xf) : measure_distant(L, P.d, P.lambda, P.s_ray2);
    add_vec(W.result, W.ns, col, m);
    return;
  }
  // every class wavelength, balance heuristic over the class
  double den = 0.0;
  for (int g = 0; g < H.G; ++g) den += H.cf[g] * H.q[g];
  for (int g = 0; g < H.G; ++g) {
    if (H.cf[g] * H.q[g] == 0.0) continue;
    const double kg = 2.0 * PI / H.lam[g];
    const double s2g = 1.0 / (2.0 * W.beta0 * W.beta0 * kg * kg);  // the invariant spread at lambda_g
    double m = 0.0;
    for (const Light& L : W.S.lights) m += measure_distant(L, P.d, H.lam[g], s2g);
    add_vec(W.result + 4 * g, W.ns, col, m * H.cf[g] * H.q[g] / den);
  }
}

// --- measurement of an emissive triangle hit at x (Eq. measurement_operator,
// footprint-sampled), weighted against next-event estimation by MIS when the
// last direction came from a diffuse rough lobe
void measure_emitter_hit(Sample& W, int seg, int prim, V3 x, const double* col) {
  const PathState& P = W.P;
  const HeroClass& H = W.H;
  const Tri& T = W.S.tris[prim];
  const Material& M = W.S.mats[T.mat];
  double u[4];
  W.rng.draw(seg, CALL_EMIT_FOOT, u);
  const bool two = (W.C.flags & FLAG_NEE) && !P.prev_delta && W.n_emit > 0;
  if (H.on) {
    const V3 ne = tri_normal(T);
    const double pb = P.prev_pdf;  // the hero's lobe density of the last direction
    // with two techniques, cf_j qpre_j p_{j,lobe} = cf_j q_j pb (q = qpre times
    // the lobe density ratio of the last vertex)
    double den = 0.0;
    for (int j = 0; j < H.G; ++j) {
      if (two) {
        const double a = H.cf[j] * H.q[j] * pb, b = H.cf[j] * H.qpre[j] * W.nee_density(j, P.d, ne, M.coh_len_um);
        den += a * a + b * b;
      } else {
        den += H.cf[j] * H.q[j];
      }
    }
    for (int g = 0; g < H.G; ++g) {
      if (H.cf[g] * H.q[g] == 0.0 || den == 0.0) continue;
      const double m = measure_emitter(W.S, prim, x, P.d, H.b2[g], H.rho[g], H.k[g], H.lam[g], u[0], u[1]);
      const double w = two ? H.cf[g] * H.cf[H.gh] * H.q[g] * pb * pb / den : H.cf[g] * H.q[g] / den;
      add_vec(W.result + 4 * g, W.ns, col, m * w);
    }
    return;
  }
  double m = W.aniso ? measure_emitter_aniso(W.S, prim, x, P.d, W.K, P.xf, P.k, P.lambda, u[0], u[1])
                     : measure_emitter(W.S, prim, x, P.d, P.beta2, P.rho, P.k, P.lambda, u[0], u[1]);
  double w = 1.0;
  if (two) {
    V3 ne = tri_normal(T);
    double kap = 1.0 / (P.s_ray2 + source_spread2(P.lambda, M.coh_len_um));
    double pn = vmf(neg(P.d), ne, kap) / W.n_emit;
    double pb = P.prev_pdf;
    w = pb * pb / (pb * pb + pn * pn);  // power heuristic
  }
  add_vec(W.result, W.ns, col, m * w);
}

// --- Russian roulette before interaction seg+1 once 3 interactions are done
// (R14); false ends the path
bool russian_roulette(Sample& W, int seg) {
  if (!(W.C.flags & FLAG_RR) || seg < 3) return true;
  PathState& P = W.P;
  double q = std::min(1.0, std::max(0.05, W.ns == 1 ? P.t : P.T.m[0][0]));
  double u[4];
  W.rng.draw(seg, CALL_RR, u);
  if (u[0] >= q) return false;
  if (W.ns == 1)
    P.t /= q;
  else
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) P.T.m[i][j] /= q;
  return true;
}

// A surface vertex of the path, as the interaction sees it (wavevector
// reversed, Eq. action_time_reversal): the normal oriented against the
// arriving direction, the Fresnel weight and the throughput it gives.
struct Vertex {
  int prim;
  const Tri* T;
  const Material* M;
  V3 x, n, d_in, t_mir, s_o;
  double cos_i;
  V3 d_dielectric;   // a dielectric's chosen direction (reflected or refracted)
  double eta_next;   // the medium index after the vertex
  M4 TRM;            // throughput x frame rotation x Fresnel weight
  double t_new;      // the scalar throughput after the vertex
  double c_nee[4];   // the throughput column a next-event estimate carries
};

// Fresnel weight (Eq. K_reflection_refraction), as a Mueller matrix in the
// s-p frames at the incidence angle of the arriving ray; diffractive lobes are
// scaled by the same matrix (reading R12).  A dielectric chooses reflection or
// refraction with the unpolarised reflectance R (R23).
void interaction_weight(Sample& W, int seg, Vertex& X) {
  const PathState& P = W.P;
  const Material& M = *X.M;
  M4 MF = m4_identity();
  X.d_dielectric = X.d_in;
  X.eta_next = P.eta;
  if (M.type == MAT_DIELECTRIC) {
    // the front (counter-clockwise) face looks out into air; reflection or
    // refraction is chosen with the unpolarised reflectance R, and the
    // Mueller weight divided by the choice's probability; a refracted
    // radiance carries (eta_a / eta_b)^2 (camera side over light side)
    const double eta_m = M.n_re + M.cauchy_b_um2 / (P.lambda * P.lambda);
    const bool entering = dot(P.d, tri_normal(*X.T)) < 0.0;
    const double eta_a = entering ? 1.0 : eta_m, eta_b = entering ? eta_m : 1.0;
    const double n_rel = eta_b / eta_a;
    Dielectric D;
    fresnel_dielectric(X.cos_i, n_rel, &D);
    double u[4];
    W.rng.draw(seg, CALL_LOBE, u);
    if (u[0] < D.R) {
      MF = mueller_diag(D.rs, D.rp);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) MF.m[i][j] /= D.R;
      X.d_dielectric = X.d_in + (2.0 * X.cos_i) * X.n;
    } else {
      MF = mueller_diag(cplx(D.ts, 0.0), cplx(D.tp, 0.0));
      const double f = (n_rel * D.cos_t / X.cos_i) * (eta_a / eta_b) * (eta_a / eta_b) / (1.0 - D.R);
      for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) MF.m[i][j] *= f;
      X.d_dielectric = refract_dir(X.d_in, X.n, n_rel, X.cos_i, D.cos_t);
      X.eta_next = eta_b;
    }
  } else if (M.fresnel == 1) {
    cplx rs, rp;
    fresnel_conductor(X.cos_i, M.n_re, M.n_im, &rs, &rp);
    MF = mueller_diag(rs, rp);
  }
  // frame of the outgoing light of the forward problem (propagation -d_in)
  V3 k_o = neg(X.d_in);
  X.s_o = s_vector(X.n, k_o, P.xf);
  V3 p_o = cross(k_o, X.s_o);
  M4 Rot = stokes_rotation(frame_angle(X.s_o, p_o, P.xf));  // frame o -> current frame
  X.TRM = m4_mul(m4_mul(P.T, Rot), MF);
  X.t_new = P.t * MF.m[0][0];
  if (W.ns == 1)
    X.c_nee[0] = X.t_new;
  else
    for (int i = 0; i < 4; ++i) X.c_nee[i] = X.TRM.m[i][0];
}

// The sampled child ray of a vertex.
struct Lobe {
  V3 d_out;
  bool delta = true;   // a delta lobe (grating order, mirror, specular term, dielectric)
  double pdf = 0.0;    // the diffuse lobe's density of d_out (solid angle)
  bool alive = true;   // false: the sample landed on an evanescent direction
  double g_r = 0.0;    // rough surface: roughness g = (2 k sigma_h cos)^2
  double m_rough = -1.0;           // rough surface: the Poisson term drawn
  V3 delta_rough = v3(0.0, 0.0, 0.0);  // rough surface: the tangential offset drawn
};

// --- sample the scattered distribution (Eq. MC_light_transport_Q1): one
// grating order (Eq. K_grating), the mirror direction, the dielectric's
// choice, or a rough-surface term and offset (R11).  Returns false where no
// order carries energy (the path ends).  With hero MIS a grating order
// updates the class's density ratios here (R24).
bool sample_lobe(Sample& W, int seg, const Vertex& X, Lobe& L) {
  const PathState& P = W.P;
  const Material& M = *X.M;
  HeroClass& H = W.H;
  double u[4];
  W.rng.draw(seg, CALL_LOBE, u);
  if (M.type == MAT_GRATING) {
    Lobes O;
    grating_lobes(M, X.d_in, X.n, P.lambda, !(W.C.flags & FLAG_NO_RENORM), &O);
    if (O.n == 0) return false;
    // first order (ascending j) whose cumulative weight exceeds u * total
    double target = u[0] * O.total;
    double cum = 0.0;
    int pick = -1;
    for (int i = 0; i < O.n; ++i) {
      cum += O.w[i];
      if (cum > target) {
        pick = i;
        break;
      }
    }
    if (pick < 0) return false;  // only possible without renormalisation
    L.d_out = O.dir[pick];
    if (H.on) {
      if (O.order[pick] != 0) {
        H.drop_companions();  // the order's direction depends on lambda
      } else {
        // specular order: same direction at every wavelength, probability
        // a_0 / total there
        const double ph = O.w[pick] / O.total;
        for (int g = 0; g < H.G; ++g) {
          if (g == H.gh || H.q[g] == 0.0) continue;
          Lobes Lg;
          grating_lobes(M, X.d_in, X.n, H.lam[g], !(W.C.flags & FLAG_NO_RENORM), &Lg);
          double p0 = 0.0;
          for (int i = 0; i < Lg.n; ++i)
            if (Lg.order[i] == 0) p0 = Lg.w[i] / Lg.total;
          H.q[g] *= p0 / ph;
        }
      }
    }
  } else if (M.type == MAT_MIRROR) {
    L.d_out = X.d_in + (2.0 * X.cos_i) * X.n;
  } else if (M.type == MAT_DIELECTRIC) {
    L.d_out = X.d_dielectric;  // chosen by interaction_weight with the same uniform
  } else {  // MAT_ROUGH
    L.g_r = std::pow(2.0 * P.k * M.sigma_h_um * X.cos_i, 2);
    double m;
    if (L.g_r > G_CONT) {
      m = L.g_r;
    } else {
      // Poisson(g) by sequential inversion: first m with CDF(m) > u
      double p = std::exp(-L.g_r), cdf = p;
      int mi = 0;
      while (u[0] >= cdf && mi < 1000) {
        ++mi;
        p *= L.g_r / mi;
        cdf += p;
      }
      m = mi;
    }
    L.m_rough = m;
    if (m == 0.0) {
      L.d_out = X.d_in + (2.0 * X.cos_i) * X.n;
    } else {
      L.delta = false;
      double kl = P.k * M.corr_len_um;
      double sig = std::sqrt(2.0 * m / (kl * kl));
      double z0, z1;
      box_muller(u[1], u[2], &z0, &z1);
      V3 e1, e2;
      onb(X.n, &e1, &e2);
      V3 delta_t = (sig * z0) * e1 + (sig * z1) * e2;
      L.delta_rough = delta_t;
      V3 t_out = X.t_mir + delta_t;
      double tt = dot(t_out, t_out);
      if (tt >= 1.0) {
        L.alive = false;  // evanescent: no propagating energy
      } else {
        L.d_out = t_out + std::sqrt(1.0 - tt) * X.n;
        L.pdf = rough_diffuse_density(L.g_r, P.k, M.corr_len_um, delta_t) * std::sqrt(1.0 - tt);
      }
    }
  }
  return true;
}

// --- hero MIS: the class wavelengths' densities of the rough-lobe term just
// sampled (the specular term's probability e^-g, or the diffuse density at the
// sampled offset; the cosine factor is common), and the companions dropped at
// a dispersive dielectric (R24)
void hero_vertex_ratios(Sample& W, const Vertex& X, const Lobe& L) {
  const PathState& P = W.P;
  const Material& M = *X.M;
  HeroClass& H = W.H;
  if (L.alive && M.type == MAT_ROUGH) {
    for (int g = 0; g < H.G; ++g) {
      if (g == H.gh || H.q[g] == 0.0) continue;
      const double kg = 2.0 * PI / H.lam[g];
      const double gg = std::pow(2.0 * kg * M.sigma_h_um * X.cos_i, 2);
      if (L.m_rough == 0.0)  // specular term: probability e^{-g} (none in the continuous limit)
        H.q[g] *= gg > G_CONT ? 0.0 : std::exp(L.g_r - gg);
      else  // diffuse terms: density at the sampled offset (the cos factor is common)
        H.q[g] *= rough_diffuse_density(gg, kg, M.corr_len_um, L.delta_rough) /
                  rough_diffuse_density(L.g_r, P.k, M.corr_len_um, L.delta_rough);
    }
  }
  if (M.type == MAT_DIELECTRIC && M.cauchy_b_um2 != 0.0) H.drop_companions();
}

// --- next-event estimation toward an emissive triangle (rough lobes only:
// grating orders and mirror reflection are delta lobes; R21): a direction from
// the vMF of the chosen emitter's measured lobe, a shadow ray that must reach
// that emitter first, and the power heuristic against the rough lobe
void next_event(Sample& W, int seg, const Vertex& X, const Lobe& L) {
  const Material& M = *X.M;
  if (M.type != MAT_ROUGH || !(W.C.flags & FLAG_NEE) || W.n_emit <= 0) return;
  const PathState& P = W.P;
  const HeroClass& H = W.H;
  const Scene& S = W.S;
  const int n_emit = W.n_emit;
  double un[4], uf[4];
  W.rng.draw(seg, CALL_NEE_DIR, un);
  int ei = std::min(n_emit - 1, (int)(un[0] * n_emit));
  const Tri& ET = S.tris[S.emitters[ei][0]];
  const int emat = ET.mat;
  const Material& EM = S.mats[emat];
  V3 ne = tri_normal(ET);
  double kap = 1.0 / (P.s_ray2 + source_spread2(P.lambda, EM.coh_len_um));
  V3 w = vmf_sample(neg(ne), kap, un[1], un[2]);
  double cos_o = dot(w, X.n);
  if (cos_o <= 0.0) return;
  double ts;
  int sp;
  if (!(closest_hit(S, X.x, w, X.prim, true, &ts, &sp) && S.tris[sp].mat == emat)) return;
  V3 delta_t = (w - dot(w, X.n) * X.n) - X.t_mir;
  double f = (L.g_r > 0.0 ? rough_diffuse_density(L.g_r, P.k, M.corr_len_um, delta_t) : 0.0) * cos_o;
  double pn = vmf(w, neg(ne), kap) / n_emit;
  if (H.on && pn > 0.0) {
    // joint power heuristic over (class wavelength, technique); the lobe
    // density toward w at wavelength j (the cos factor included)
    double pbw[4], den = 0.0;
    for (int j = 0; j < H.G; ++j) {
      pbw[j] = 0.0;
      if (H.cf[j] * H.qpre[j] == 0.0) continue;
      const double gj = std::pow(2.0 * H.k[j] * M.sigma_h_um * X.cos_i, 2);
      pbw[j] = (gj > 0.0 ? rough_diffuse_density(gj, H.k[j], M.corr_len_um, delta_t) : 0.0) * cos_o;
      const double a = H.cf[j] * H.qpre[j] * pbw[j], b = H.cf[j] * H.qpre[j] * W.nee_density(j, w, ne, EM.coh_len_um);
      den += a * a + b * b;
    }
    W.rng.draw(seg, CALL_NEE_FOOT, uf);
    for (int g = 0; g < H.G; ++g) {
      if (pbw[g] == 0.0 || den == 0.0) continue;
      double b2 = H.b2[g], r = H.rho[g];
      propagate(&b2, &r, ts * 1e6 / (H.k[g] * P.eta));
      double m = measure_emitter(S, sp, X.x + ts * w, w, b2, r, H.k[g], H.lam[g], uf[0], uf[1]);
      add_vec(W.result + 4 * g, W.ns, X.c_nee, m * H.cf[g] * H.cf[H.gh] * H.qpre[g] * pn * pbw[g] / den);
    }
  } else if (f > 0.0 && pn > 0.0 && W.aniso) {
    // the vertex's footprint mapped to the emitter direction's frame
    const V3 xf_w = s_vector(X.n, neg(w), X.s_o);
    CS2 Kw = aniso_interaction(W.K, P.xf, X.d_in, xf_w, w, X.n);
    aniso_propagate(&Kw, ts * 1e6 / (P.k * P.eta));
    W.rng.draw(seg, CALL_NEE_FOOT, uf);
    double m = measure_emitter_aniso(S, sp, X.x + ts * w, w, Kw, xf_w, P.k, P.lambda, uf[0], uf[1]);
    double wmis = pn * pn / (pn * pn + f * f);
    add_vec(W.result, W.ns, X.c_nee, m * f / pn * wmis);
  } else if (f > 0.0 && pn > 0.0) {
    double b2 = P.beta2, r = P.rho;
    propagate(&b2, &r, ts * 1e6 / (P.k * P.eta));
    W.rng.draw(seg, CALL_NEE_FOOT, uf);
    double m = measure_emitter(S, sp, X.x + ts * w, w, b2, r, P.k, P.lambda, uf[0], uf[1]);
    double wmis = pn * pn / (pn * pn + f * f);
    add_vec(W.result, W.ns, X.c_nee, m * f / pn * wmis);
  }
}

// --- continue the path with the sampled generalized ray: position and
// (beta, rho) unchanged by the interaction (Eq. K_reflection_refraction; rho
// growth at the grating ignored, Eq. K_grating); the anisotropic footprint is
// mapped onto the outgoing direction's frame (R25)
void continue_path(Sample& W, const Vertex& X, const Lobe& L) {
  PathState& P = W.P;
  if (W.aniso) {
    const V3 xf_out = s_vector(X.n, neg(L.d_out), X.s_o);
    W.K = aniso_interaction(W.K, P.xf, X.d_in, xf_out, L.d_out, X.n);
    P.xf = xf_out;
  }
  if (W.ns == 1) {
    P.t = X.t_new;
  } else {
    P.T = X.TRM;
    V3 k_i = neg(L.d_out);
    P.xf = s_vector(X.n, k_i, X.s_o);
  }
  P.o = X.x;
  P.d = L.d_out;
  P.eta = X.eta_next;
  P.prev_prim = X.prim;
  P.prev_delta = L.delta;
  P.prev_pdf = L.pdf;
}

// One path sample of pixel (px, py), Algorithm 1 with the interactive
// simplifications of Sec. 7.2: source, then per segment propagate (closest
// hit, footprint update), measure (escape or emitter hit: the path ends),
// Russian roulette, interact (weight, sampled child ray), next-event estimate,
// continue.  result: the sample's contribution [Stokes] (with hero MIS
// [class bin][Stokes]).
void trace_sample(const Ctx& C, int px, int py, long sample, double* result) {
  Sample W(C, result);
  source(W, px, py, sample);
  PathState& P = W.P;
  HeroClass& H = W.H;
  for (int seg = 0;; ++seg) {
    // --- propagation: closest hit along d (point-hit assumption, Sec. 7.2)
    double th;
    int prim;
    bool hit = closest_hit(W.S, P.o, P.d, P.prev_prim, true, &th, &prim);
    double col[4];
    throughput_column(P, W.ns, col);
    if (!hit) {
      measure_escape(W, col);
      return;
    }
    // footprint update over the segment (z in um; |k| = eta k0 in a medium;
    // Eq. K_free_space_propagation)
    propagate(&P.beta2, &P.rho, th * 1e6 / (P.k * P.eta));
    if (W.aniso) aniso_propagate(&W.K, th * 1e6 / (P.k * P.eta));
    if (H.on)
      for (int g = 0; g < H.G; ++g) propagate(&H.b2[g], &H.rho[g], th * 1e6 / (H.k[g] * P.eta));
    V3 x = P.o + th * P.d;
    const Tri& T = W.S.tris[prim];
    const Material& M = W.S.mats[T.mat];
    if (M.type == MAT_EMITTER) {
      measure_emitter_hit(W, seg, prim, x, col);
      return;
    }
    if (M.type == MAT_ABSORBER) return;
    if (seg >= W.V.max_depth) return;  // no interactions left
    if (!russian_roulette(W, seg)) return;

    // --- light-matter interaction with the wavevector reversed (Eq.
    // action_time_reversal): the surface normal is oriented against d.
    Vertex X;
    X.prim = prim;
    X.T = &T;
    X.M = &M;
    X.x = x;
    X.n = tri_normal(T);
    if (dot(X.n, P.d) > 0.0) X.n = neg(X.n);
    X.cos_i = -dot(P.d, X.n);
    X.d_in = P.d;
    X.t_mir = X.d_in - dot(X.d_in, X.n) * X.n;
    for (int g = 0; g < H.G; ++g) H.qpre[g] = H.q[g];
    interaction_weight(W, seg, X);
    Lobe L;
    if (!sample_lobe(W, seg, X, L)) return;
    if (H.on) hero_vertex_ratios(W, X, L);
    next_event(W, seg, X, L);
    if (!L.alive) return;
    continue_path(W, X, L);
  }
}
}  // namespace

// ======================================================================= C ABI
extern "C" {

int oracle_abi_version() { return 1; }

// Dielectric interface at cos_i with relative index n_rel (test access):
// out = [Rs, Rp, Ts, Tp, R, T, cos_t, tir].
void oracle_fresnel_dielectric(double cos_i, double n_rel, double* out) {
  Dielectric D;
  fresnel_dielectric(cos_i, n_rel, &D);
  const double f = D.tir ? 0.0 : n_rel * D.cos_t / cos_i;
  out[0] = std::norm(D.rs);
  out[1] = std::norm(D.rp);
  out[2] = f * D.ts * D.ts;
  out[3] = f * D.tp * D.tp;
  out[4] = D.R;
  out[5] = D.T;
  out[6] = D.cos_t;
  out[7] = D.tir ? 1.0 : 0.0;
}

// Refracted direction for incidence d at a surface with normal n (either
// orientation) from index eta_a into eta_b (test access); returns 0 under total
// internal reflection.
int oracle_refract(const double* d, const double* n, double eta_a, double eta_b, double* out) {
  V3 dd = v3(d[0], d[1], d[2]), nn = v3(n[0], n[1], n[2]);
  if (dot(dd, nn) > 0.0) nn = neg(nn);
  const double cos_i = -dot(dd, nn);
  Dielectric D;
  fresnel_dielectric(cos_i, eta_b / eta_a, &D);
  if (D.tir) return 0;
  V3 t = refract_dir(dd, nn, eta_b / eta_a, cos_i, D.cos_t);
  out[0] = t.x;
  out[1] = t.y;
  out[2] = t.z;
  return 1;
}


void oracle_philox4x32_10(const uint32_t* ctr, const uint32_t* key, uint32_t* out) { philox4x32_10(ctr, key, out); }

double oracle_bessel_j(int n, double x) { return bessel_j(n, x); }

double oracle_vmf(const double* w, const double* mu, double kappa) {
  return vmf(v3(w[0], w[1], w[2]), v3(mu[0], mu[1], mu[2]), kappa);
}

void oracle_vmf_sample(const double* mu, double kappa, double u0, double u1, double* out) {
  V3 r = vmf_sample(v3(mu[0], mu[1], mu[2]), kappa, u0, u1);
  out[0] = r.x;
  out[1] = r.y;
  out[2] = r.z;
}

void oracle_onb(const double* n, double* e1, double* e2) {
  V3 a, b;
  onb(v3(n[0], n[1], n[2]), &a, &b);
  e1[0] = a.x; e1[1] = a.y; e1[2] = a.z;
  e2[0] = b.x; e2[1] = b.y; e2[2] = b.z;
}

void oracle_propagate(double beta2, double rho, double zbar, double* out) {
  propagate(&beta2, &rho, zbar);
  out[0] = beta2;
  out[1] = rho;
}

// Material parameter vector (float32[16]) and light vector (float32[8]) layout:
// see oracle/oracle.py.
static Material read_material(const float* m) {
  Material M;
  M.type = (int)m[0];
  M.fresnel = (int)m[1];
  M.n_re = m[2];
  M.n_im = m[3];
  M.period_um = m[4];
  M.height_um = m[5];
  M.gdir = v3(m[6], m[7], m[8]);
  M.sigma_h_um = m[9];
  M.corr_len_um = m[10];
  M.Le = m[11];
  M.coh_len_um = m[12];
  M.cauchy_b_um2 = m[13];
  return M;
}

// Grating lobes for one incidence (test access).  Returns the number of
// propagating orders written (orders[i], weights[i] normalised by the total,
// dirs[3i..3i+2]).
int oracle_grating_lobes(const float* mat, const double* d_in, const double* n, double lambda_um, int renorm,
                         int cap, int* orders, double* weights, double* dirs) {
  Material M = read_material(mat);
  Lobes L;
  grating_lobes(M, v3(d_in[0], d_in[1], d_in[2]), v3(n[0], n[1], n[2]), lambda_um, renorm != 0, &L);
  int k = std::min(cap, L.n);
  for (int i = 0; i < k; ++i) {
    orders[i] = L.order[i];
    weights[i] = L.w[i] / L.total;
    dirs[3 * i] = L.dir[i].x;
    dirs[3 * i + 1] = L.dir[i].y;
    dirs[3 * i + 2] = L.dir[i].z;
  }
  return L.n;
}

double oracle_rough_density(double g, double k, double ell, double dx, double dy) {
  return rough_diffuse_density(g, k, ell, v3(dx, dy, 0.0));
}

void oracle_fresnel_mueller(double cos_i, double n_re, double n_im, double* out16, double* rs_rp4) {
  cplx rs, rp;
  fresnel_conductor(cos_i, n_re, n_im, &rs, &rp);
  M4 M = mueller_diag(rs, rp);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) out16[4 * i + j] = M.m[i][j];
  if (rs_rp4) {
    rs_rp4[0] = rs.real();
    rs_rp4[1] = rs.imag();
    rs_rp4[2] = rp.real();
    rs_rp4[3] = rp.imag();
  }
}

void oracle_stokes_rotation(double phi, double* out16) {
  M4 M = stokes_rotation(phi);
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) out16[4 * i + j] = M.m[i][j];
}

void* oracle_scene_create(int n_tris, const float* verts, const int* tri_mat, int n_mats, const float* mats,
                          int n_lights, const float* lights) {
  Scene* S = new Scene();
  S->tris.resize(n_tris);
  for (int i = 0; i < n_tris; ++i) {
    const float* v = verts + 9 * i;
    S->tris[i].v0 = v3(v[0], v[1], v[2]);
    S->tris[i].v1 = v3(v[3], v[4], v[5]);
    S->tris[i].v2 = v3(v[6], v[7], v[8]);
    S->tris[i].mat = tri_mat[i];
  }
  for (int i = 0; i < n_mats; ++i) S->mats.push_back(read_material(mats + 16 * i));
  for (int i = 0; i < n_lights; ++i) {
    const float* l = lights + 8 * i;
    Light L;
    L.type = (int)l[0];
    L.dir = v3(l[1], l[2], l[3]);
    if (L.type == 0) L.dir = normalize(L.dir);
    L.E = l[4];
    L.coh_len_um = l[5];
    S->lights.push_back(L);
  }
  S->emitter_of_mat.assign(n_mats, -1);
  for (int i = 0; i < n_tris; ++i) {
    int m = S->tris[i].mat;
    if (S->mats[m].type != MAT_EMITTER) continue;
    if (S->emitter_of_mat[m] < 0) {
      S->emitter_of_mat[m] = (int)S->emitters.size();
      S->emitters.push_back(std::vector<int>());
    }
    S->emitters[S->emitter_of_mat[m]].push_back(i);
  }
  if (n_tris > 0) {
    S->order.resize(n_tris);
    for (int i = 0; i < n_tris; ++i) S->order[i] = i;
    build_bvh(*S, 0, n_tris);
  }
  return S;
}

void oracle_scene_destroy(void* s) { delete (Scene*)s; }

// Traversal work since the last reset: out[0] closest-hit queries, out[1]
// internal node visits, out[2] ray-triangle tests (summed over threads).
void oracle_work_counters(long long* out) {
  out[0] = g_work_queries.load();
  out[1] = g_work_visits.load();
  out[2] = g_work_tests.load();
}

void oracle_work_reset(void) {
  g_work_queries = 0;
  g_work_visits = 0;
  g_work_tests = 0;
}

int oracle_closest_hit(void* s, const double* o, const double* d, int exclude, int use_bvh, double* t, int* prim) {
  Scene* S = (Scene*)s;
  double tt = 0.0;
  int pp = -1;
  bool h = closest_hit(*S, v3(o[0], o[1], o[2]), v3(d[0], d[1], d[2]), exclude, use_bvh != 0, &tt, &pp);
  *t = h ? tt : -1.0;
  *prim = h ? pp : -1;
  return h ? 1 : 0;
}

// View parameter vector (double[24]):
//  0-2 eye, 3-5 look_at, 6-8 up, 9 vfov_deg, 10 W, 11 H, 12 p_pix_um, 13 f_beta,
//  14 lambda_min_um, 15 lambda_max_um, 16 n_bins, 17 n_stokes, 18 max_depth,
//  19 spp, 20 first_sample, 21 view_index, 22 ortho (0/1), 23 ortho half height (m)
static View read_view(const double* p) {
  View V;
  V.eye = v3(p[0], p[1], p[2]);
  V.look = v3(p[3], p[4], p[5]);
  V.up = v3(p[6], p[7], p[8]);
  V.vfov_deg = p[9];
  V.W = (int)p[10];
  V.H = (int)p[11];
  V.p_pix_um = p[12];
  V.f_beta = p[13];
  V.lmin_um = p[14];
  V.lmax_um = p[15];
  V.n_bins = (int)p[16];
  V.n_stokes = (int)p[17];
  V.max_depth = (int)p[18];
  V.spp = (long)p[19];
  V.first_sample = (long)p[20];
  V.view_index = (uint32_t)p[21];
  V.ortho = (int)p[22];
  V.ortho_half_m = p[23];
  return V;
}

// One path sample's contribution for tests: out16[4 g + k], class bin g (only
// g = 0 without hero MIS), Stokes component k.
// Anisotropic footprint maps for tests; K as 6 doubles (Re, Im) of K11, K12,
// K22.  Free-space propagation by zbar (um), and the interaction map for the
// frames (f_in, d_in) -> (f_out, d_out) at a surface of normal n.
void oracle_aniso_propagate(const double* k6, double zbar, double* out6) {
  CS2 K{cplx(k6[0], k6[1]), cplx(k6[2], k6[3]), cplx(k6[4], k6[5])};
  aniso_propagate(&K, zbar);
  const cplx r[3] = {K.a, K.b, K.c};
  for (int i = 0; i < 3; ++i) out6[2 * i] = r[i].real(), out6[2 * i + 1] = r[i].imag();
}
void oracle_aniso_interaction(const double* k6, const double* f_in, const double* d_in, const double* f_out,
                              const double* d_out, const double* n, double* out6) {
  CS2 K{cplx(k6[0], k6[1]), cplx(k6[2], k6[3]), cplx(k6[4], k6[5])};
  auto V = [](const double* a) { return v3(a[0], a[1], a[2]); };
  CS2 R = aniso_interaction(K, V(f_in), V(d_in), V(f_out), V(d_out), V(n));
  const cplx r[3] = {R.a, R.b, R.c};
  for (int i = 0; i < 3; ++i) out6[2 * i] = r[i].real(), out6[2 * i + 1] = r[i].imag();
}

// The footprint point, its direction shift and the emitter lobe (unit
// exitance, point covered) for the standard normal pair (z0, z1); out6 =
// x1, x2 (um, frame onb(d)), m1, m2, lobe value, 0.
void oracle_aniso_emitter(const double* k6, const double* xf, const double* d, double k, double s2, const double* ne,
                          double z0, double z1, double* out6) {
  CS2 K{cplx(k6[0], k6[1]), cplx(k6[2], k6[3]), cplx(k6[4], k6[5])};
  const V3 dd = v3(d[0], d[1], d[2]);
  const AnisoFoot F = aniso_footprint(dd, K, v3(xf[0], xf[1], xf[2]), k, z0, z1);
  out6[0] = F.x1;
  out6[1] = F.x2;
  out6[2] = F.m1;
  out6[3] = F.m2;
  out6[4] = aniso_emitter_lobe(F, dd, k, s2, v3(ne[0], ne[1], ne[2]));
  out6[5] = 0.0;
}

void oracle_trace_sample(void* s, const double* view, uint32_t seed, int flags, int px, int py, long sample,
                         double* out16) {
  Scene* S = (Scene*)s;
  View V = read_view(view);
  Ctx C;
  C.S = S;
  C.V = &V;
  C.flags = flags;
  C.rng.key[0] = seed;
  C.rng.key[1] = V.view_index;
  trace_sample(C, px, py, sample, out16);
}

// Render the pixels of the crop [x0,x1) x [y0,y1): for every pixel and bin, the
// mean over the samples s in [first_sample, first_sample + spp) with
// s mod n_bins == bin, summed in sample order with compensated (Neumaier)
// summation.  With FLAG_HERO (n_bins a multiple of 4) every sample also adds
// its weighted contributions to the other bins of its class, and a bin's
// sum is still divided by the number of samples whose hero it is (the
// weights make that the class average); out_var then holds the second moment
// of the added values about that mean, not a per-sample variance.  Returns -1
// for FLAG_HERO with n_bins not a multiple of 4.  out_mean: [crop_h][crop_w][n_bins][n_stokes]; out_var (optional):
// the per-sample variance of the same values.  Returns the number of samples.
long oracle_render(void* s, const double* view, uint32_t seed, int flags, int x0, int y0, int x1, int y1,
                   int n_threads, double* out_mean, double* out_var) {
  Scene* S = (Scene*)s;
  View V = read_view(view);
  if ((flags & FLAG_HERO) && V.n_bins % 4 != 0) return -1;  // hero classes need 4 | n_bins
  if ((flags & FLAG_HERO) && (flags & FLAG_ANISO)) return -2;  // not combined
  Ctx C;
  C.S = S;
  C.V = &V;
  C.flags = flags;
  C.rng.key[0] = seed;
  C.rng.key[1] = V.view_index;
  const int cw = x1 - x0, ch = y1 - y0;
  const int nb = V.n_bins, ns = V.n_stokes;
  std::atomic<int> next_row(0);
  auto worker = [&]() {
    std::vector<double> sum(nb * 4), comp(nb * 4), sq(nb * 4);
    std::vector<long> cnt(nb);
    for (;;) {
      int r = next_row.fetch_add(1);
      if (r >= ch) break;
      int py = y0 + r;
      for (int px = x0; px < x1; ++px) {
        std::fill(sum.begin(), sum.end(), 0.0);
        std::fill(comp.begin(), comp.end(), 0.0);
        std::fill(sq.begin(), sq.end(), 0.0);
        std::fill(cnt.begin(), cnt.end(), 0L);
        for (long si = 0; si < V.spp; ++si) {
          long smp = V.first_sample + si;
          double c[16];
          trace_sample(C, px, py, smp, c);
          int b = (int)(smp % nb);
          cnt[b]++;
          // without hero MIS the sample adds to its bin; with it, to each bin
          // of its class (c[4 g + k] for class bin g)
          const int G = (flags & FLAG_HERO) ? 4 : 1, Qb = nb / G, c0 = b % Qb;
          for (int g = 0; g < G; ++g) {
            const int bb = G == 1 ? b : c0 + g * Qb;
            for (int k = 0; k < ns; ++k) {
              // Neumaier compensated summation
              double a = sum[bb * 4 + k], v = c[4 * g + k];
              double t = a + v;
              if (std::fabs(a) >= std::fabs(v))
                comp[bb * 4 + k] += (a - t) + v;
              else
                comp[bb * 4 + k] += (v - t) + a;
              sum[bb * 4 + k] = t;
              sq[bb * 4 + k] += v * v;
            }
          }
        }
        size_t base = ((size_t)r * cw + (px - x0)) * nb * ns;
        for (int b = 0; b < nb; ++b)
          for (int k = 0; k < ns; ++k) {
            double tot = sum[b * 4 + k] + comp[b * 4 + k];
            double mean = cnt[b] ? tot / cnt[b] : 0.0;
            out_mean[base + b * ns + k] = mean;
            if (out_var) out_var[base + b * ns + k] = cnt[b] ? sq[b * 4 + k] / cnt[b] - mean * mean : 0.0;
          }
      }
    }
  };
  int nt = std::max(1, n_threads);
  std::vector<std::thread> th;
  for (int i = 0; i < nt; ++i) th.emplace_back(worker);
  for (auto& t : th) t.join();
  return (long)cw * ch * V.spp;
}

}  // extern "C"
