// Wavefront integrator for backward path tracing of generalized rays.
//
// Work decomposition.  A ticket is one (view, spectral bin, pixel); it owns the
// samples s in [first_sample, first_sample + spp) with s mod n_bins == bin,
// which one pool slot traces one after another and sums (Kahan) in sample
// order, so every pixel value is deterministic whatever the schedule.  A fixed
// pool of P slots persists across iterations; each iteration is four kernels:
//   regen  : fold finished samples, start the ticket's next sample (camera
//            generalized ray, Eq. MC_sourcing), or claim new tickets with one
//            warp-aggregated atomic per warp; compact live slots into the
//            trace queue (ballot + popc)
//   trace  : closest hit of every queued ray and of the previous shade's
//            next-event rays, in one load-balanced launch (BVH, stack
//            traversal)
//   shadow : measure the emitter each next-event ray reached and add the
//            MIS-weighted contribution (before the segment's own shading, so
//            the sample's terms are added in path order); close the
//            iteration's queues
//   shade  : footprint update (Eq. K_free_space_propagation), measurement on
//            escape / emitter hit (Eq. measurement_operator), interaction with
//            the reversed wavevector (Eq. action_time_reversal) and sampling of
//            one child ray (Eq. MC_light_transport_Q1): grating orders
//            (Eq. K_grating, order tables staged in shared memory), rough lobe
//            (Eq. K_surface_HS), smooth reflection (Eq. K_reflection_refraction)
//            with Fresnel Mueller weights; NEE shadow requests are queued
// A sample that ends at a vertex with a next-event request waits (ST_WAIT)
// one regen pass for its ray, so its fold still follows its last term.
// All launches have fixed shapes (grid-stride loops over device-side queue
// counts), so a batch of iterations can be replayed as one CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "gr_build.h"

namespace gr {

// slot states; ST_WAIT: the sample has ended, but its last vertex's
// next-event ray is traced and measured in the next iteration (the slot is
// folded one regen pass later)
enum { ST_IDLE = 0, ST_ACTIVE = 1, ST_DONE = 2, ST_WAIT = 3 };
// trace-launch entries that are next-event rays carry this bit on the slot
constexpr int kShadowEntry = 1 << 30;

// Default slot pool bounds (slots; 265 bytes each without the hero and
// anisotropic planes).
constexpr long long kMaxDefaultPool = 1LL << 25;
constexpr long long kMinDefaultPool = 1LL << 16;

// Minimum resident 256-thread blocks per SM requested for the traversal
// kernels (register budget 65536 / (256 x blocks)).
// binary-tree trace kernel: 128-thread blocks, 7 per SM (<= 72 registers)
#ifndef GR_TRACE_MIN_BLOCKS
#define GR_TRACE_MIN_BLOCKS 7
#endif
#ifndef GR_TRACE_BLOCK
#define GR_TRACE_BLOCK 128
#endif
// shading: 4 blocks/SM (64 registers) for both Stokes counts.  The spills
// this costs the 4-Stokes kernel are cheaper than the latency left exposed
// with a quarter fewer resident warps (measured on both forms).
#ifndef GR_SHADE_MIN_BLOCKS
#define GR_SHADE_MIN_BLOCKS 4
#endif
#ifndef GR_SHADE_MIN_BLOCKS_NS1
#define GR_SHADE_MIN_BLOCKS_NS1 4
#endif
// the hero-wavelength instantiations at 4 blocks/SM (2 and 3 measured
// slower); the anisotropic ones at 3 (2.5% faster than 4 on the headline)
#ifndef GR_SHADE_MIN_BLOCKS_HERO
#define GR_SHADE_MIN_BLOCKS_HERO 4
#endif
#ifndef GR_SHADE_MIN_BLOCKS_ANISO
#define GR_SHADE_MIN_BLOCKS_ANISO 3
#endif

__device__ __forceinline__ int meta_k(int z) { return z & 0xffff; }
__device__ __forceinline__ int meta_seg(int z) { return (z >> 16) & 0xff; }
__device__ __forceinline__ int meta_delta(int z) { return (z >> 26) & 1; }
__device__ __forceinline__ int meta_pack(int k, int seg, int st, int delta) {
  return k | (seg << 16) | (st << 24) | (delta << 26);
}

// First sample s >= first_sample with s mod Q == c, and the number of the
// view's samples in that residue class.  A ticket owns one class: with Q = nb
// a class is one wavelength bin; with hero-wavelength MIS (Q = nb/4) the
// class's samples are heroes of the bins c, c+Q, c+2Q, c+3Q in turn.
__device__ __forceinline__ int class_first_sample(const DevView& V, int c, int Q) {
  int r = (c - V.first_sample) % Q;
  if (r < 0) r += Q;
  return V.first_sample + r;
}
__device__ __forceinline__ int class_samples(const DevView& V, int c, int Q) {
  int s0 = class_first_sample(V, c, Q);
  int end = V.first_sample + V.spp;
  return s0 < end ? (end - 1 - s0) / Q + 1 : 0;
}
__device__ __forceinline__ int bin_samples(const DevView& V, int bin) { return class_samples(V, bin, V.nb); }
// Wavelength of bin b from the bin step (lmax - lmin) / (nb - 1), computed
// once per path: the class wavelengths of hero-wavelength MIS cost one
// multiply-add each instead of a division.
__device__ __forceinline__ float bin_step(const DevView& V) {
  return V.nb <= 1 ? 0.0f : (V.lmax - V.lmin) / (float)(V.nb - 1);
}
__device__ __forceinline__ float step_lambda(const DevView& V, float step, int b) { return V.lmin + (float)b * step; }
constexpr float kInv2Pi = 0.15915494309189535f;
// cf[g]: the share of class c's samples (modulus Q) whose hero is bin c + g Q.
__device__ __forceinline__ void class_shares(const DevView& V, int c, int Q, float cf[4]) {
  const float n = (float)class_samples(V, c, Q);
#pragma unroll
  for (int g = 0; g < 4; ++g) cf[g] = (float)bin_samples(V, c + g * Q) / n;
}
__device__ __forceinline__ float bin_lambda(const DevView& V, int b) {
  if (V.nb <= 1) return V.lmin;
  return V.lmin + (float)b * (V.lmax - V.lmin) / (float)(V.nb - 1);
}
__device__ __forceinline__ double bin_lambda_d(const DevView& V, int b) {
  if (V.nb <= 1) return (double)V.lmin;
  return (double)V.lmin + (double)b * ((double)V.lmax - (double)V.lmin) / (double)(V.nb - 1);
}
// Angular variance of a source of coherence length lc (um): (lambda/lc)^2.
__device__ __forceinline__ float src_spread2(float lambda, float lc) {
  if (lc <= 0.0f) return 0.0f;
  float s = lambda / lc;
  return s * s;
}

// Entry e of the trace queue: the first `front` entries sit at the start of
// the array, the rest at its end in reverse.
__device__ __forceinline__ int tq_entry(const RenderParams& p, int e, int front) {
  return e < front ? p.pool.tq[e] : p.pool.tq[p.P - 1 - (e - front)];
}

// The view that owns ticket t: binary search over the views' first tickets,
// read from `bases` (a shared-memory copy) when given, else from the views.
__device__ __forceinline__ int find_view(const RenderParams& p, unsigned long long t,
                                         const long long* bases = nullptr) {
  int lo = 0, hi = p.n_views - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    const long long b = bases ? bases[mid] : p.views[mid].ticket_base;
    if ((unsigned long long)b <= t)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
// views whose first tickets k_regen stages in shared memory (4 KB)
#ifndef GR_REGEN_SLOTS
#define GR_REGEN_SLOTS 4
#endif
#ifndef GR_REGEN_SMEM_VIEWS
#define GR_REGEN_SMEM_VIEWS 512
#endif

template <typename TT>
__device__ __forceinline__ float table_load(const TT* v, int i);
template <>
__device__ __forceinline__ float table_load<float>(const float* v, int i) {
  return v[i];
}
template <>
__device__ __forceinline__ float table_load<__half>(const __half* v, int i) {
  return __half2float(v[i]);
}
template <>
__device__ __forceinline__ float table_load<__nv_bfloat16>(const __nv_bfloat16* v, int i) {
  return __bfloat162float(v[i]);
}

// ------------------------------------------------------------------ sourcing
template <int NS, bool HERO>
__device__ __forceinline__ void start_sample(const RenderParams& p, int slot, int view, int local, int k) {
  const DevView& V = p.views[view];
  const int WH = V.W * V.H;
  const int cls = local / WH;
  const int pixel = local - cls * WH;
  const int py = pixel / V.W, px = pixel - py * V.W;
  const int s = class_first_sample(V, cls, V.Q) + k * V.Q;
  float4 u = rng4(p.seed, (uint32_t)V.view_index, (uint32_t)pixel, (uint32_t)s, 0, kCallJitter);
  float fx = ((float)px + u.x) / (float)V.W, fy = ((float)py + u.y) / (float)V.H;
  float3 o, d;
  if (V.ortho) {
    o = V.eye + ((2.0f * fx - 1.0f) * V.ortho_half * V.aspect) * V.right + ((1.0f - 2.0f * fy) * V.ortho_half) * V.upc;
    d = V.fw;
  } else {
    float sx = (2.0f * fx - 1.0f) * V.th * V.aspect;
    float sy = (1.0f - 2.0f * fy) * V.th;
    o = V.eye;
    d = normalize(V.fw + sx * V.right + sy * V.upc);
  }
  const Pool& P = p.pool;
  P.od0[slot] = make_float4(o.x, o.y, o.z, V.beta0 * V.beta0);
  P.od1[slot] = make_float4(d.x, d.y, d.z, 0.0f);
  // the throughput (identity), the Stokes frame, the medium (air) and the
  // contribution (zero) of a camera segment are implied by segment 0: k_shade
  // forms them instead of reading them
  P.meta[slot] = make_int4(view, local, meta_pack(k, 0, ST_ACTIVE, 1), -1);
  P.st8[slot] = ST_ACTIVE;
}

// Sum a per-thread count over the warp and add it with one atomic.
__device__ __forceinline__ void warp_count(unsigned long long* ctr, int v) {
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(ctr, (unsigned long long)v);
}

// Block-wide queue reservation with one atomic per block: returns this
// thread's slot in the queue for `want` entries (exclusive scan over the
// block's warps).  Every thread of the block must call it (uniform control
// flow); the trailing barrier lets the shared words be reused by the next call.
template <typename CT>
__device__ __forceinline__ CT block_reserve(CT* counter, bool want) {
  __shared__ int s_warp[8];
  __shared__ CT s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, want);
  if (lane == 0) s_warp[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < nw; ++w) {
      const int c = s_warp[w];
      s_warp[w] = tot;
      tot += c;
    }
    s_base = tot ? atomicAdd(counter, (CT)tot) : (CT)0;
  }
  __syncthreads();
  const CT off = s_base + (CT)(s_warp[warp] + __popc(m & ((1u << lane) - 1u)));
  __syncthreads();
  return off;
}

// Two block-wide queue reservations with one set of barriers: this thread's
// entries in queue a (for want_a) and in queue b (for want_b).  Uniform
// control flow, as block_reserve.
__device__ __forceinline__ int2 block_reserve2(int* counter_a, bool want_a, int* counter_b, bool want_b) {
  __shared__ int s_wa[8], s_wb[8];
  __shared__ int s_base[2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  const unsigned ma = __ballot_sync(0xffffffffu, want_a), mb = __ballot_sync(0xffffffffu, want_b);
  if (lane == 0) {
    s_wa[warp] = __popc(ma);
    s_wb[warp] = __popc(mb);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int ta = 0, tb = 0;
    for (int w = 0; w < nw; ++w) {
      const int ca = s_wa[w], cb = s_wb[w];
      s_wa[w] = ta;
      s_wb[w] = tb;
      ta += ca;
      tb += cb;
    }
    s_base[0] = ta ? atomicAdd(counter_a, ta) : 0;
    s_base[1] = tb ? atomicAdd(counter_b, tb) : 0;
  }
  __syncthreads();
  const unsigned below = (1u << lane) - 1u;
  const int2 off = make_int2(s_base[0] + s_wa[warp] + __popc(ma & below), s_base[1] + s_wb[warp] + __popc(mb & below));
  __syncthreads();
  return off;
}

// Block-wide reservation of n entries per thread (n >= 0) with one atomic per
// block: returns the first of this thread's n entries (exclusive scan over the
// block).  Uniform control flow, as block_reserve.
template <typename CT>
__device__ __forceinline__ CT block_reserve_n(CT* counter, int n) {
  __shared__ int s_warp[8];
  __shared__ CT s_base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int incl = n;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += v;
  }
  if (lane == 31) s_warp[warp] = incl;
  __syncthreads();
  if (threadIdx.x == 0) {
    int tot = 0;
    for (int w = 0; w < nw; ++w) {
      const int c = s_warp[w];
      s_warp[w] = tot;
      tot += c;
    }
    s_base = tot ? atomicAdd(counter, (CT)tot) : (CT)0;
  }
  __syncthreads();
  const CT off = s_base + (CT)(s_warp[warp] + incl - n);
  __syncthreads();
  return off;
}

// Block-wide sum of a per-thread count added with one atomic per block.
__device__ __forceinline__ void block_count(unsigned long long* ctr, int v) {
  __shared__ int s_sum[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if (lane == 0) s_sum[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long tot = 0;
    for (int w = 0; w < nw; ++w) tot += s_sum[w];
    if (tot) atomicAdd(ctr, (unsigned long long)tot);
  }
  __syncthreads();
}

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
  float y = v - c;
  float t = s + y;
  c = (t - s) - y;
  s = t;
}

// ------------------------------------------------------------------ regen
// Hero-wavelength MIS: fold the finished sample into the ticket's four member
// sums (member g = bin c + g Q): its own contribution into the hero's member,
// its shares at the other class wavelengths (escapes, emitter hits,
// next-event estimates) into theirs.  On the ticket's last sample every
// member's total goes to its bin's frame accumulator.  Returns true if the
// ticket has more samples.
// A term of class member g's range sum (hero-wavelength MIS, g not the
// sample's hero): Kahan-added to the slot's sum as soon as it is measured,
// in path order (the hero's own terms go through the sample's contribution
// and are folded when the sample ends).  col: the throughput column.
template <int NS>
__device__ __forceinline__ void member_add(const Pool& P, size_t Ps, int g, int slot, float c0, float c1, float c2,
                                           float c3, float val) {
  float4 sm = P.haccS[g * Ps + slot], c = P.haccC[g * Ps + slot];
  kahan_add(sm.x, c.x, c0 * val);
  if (NS == 4) {
    kahan_add(sm.y, c.y, c1 * val);
    kahan_add(sm.z, c.z, c2 * val);
    kahan_add(sm.w, c.w, c3 * val);
  }
  P.haccS[g * Ps + slot] = sm;
  P.haccC[g * Ps + slot] = c;
}

// Sample ranges of a class ticket under hero-wavelength MIS: with hs > 1 the
// n samples k of a class are split into hs tickets, range j holding
// k in [floor(j n / hs), floor((j + 1) n / hs)) (never empty: n >= hs).
__device__ __forceinline__ int range_of(int k, int n, int hs) { return ((k + 1) * hs - 1) / n; }
__device__ __forceinline__ int range_begin(int j, int n, int hs) { return (j * n) / hs; }

// Fold a finished hero sample's own total into its member's range sum
// (Kahan, per Stokes component; the companions' terms are already in theirs,
// member_add); at the end of the ticket's range, add the four members' range
// totals into the frame.  With hs > 1 the ranges of a class finish in any
// order: each stores its totals in the class record, and the last to finish
// adds all of them, in range order, so every frame element still receives
// its terms in sample order whatever the schedule.  Returns true if the
// ticket has another sample.
template <int NS>
__device__ __forceinline__ bool fold_class(const RenderParams& p, int slot, const int4& m) {
  const Pool& P = p.pool;
  const DevView& V = p.views[m.x];
  const int WH = V.W * V.H;
  const int cls = m.y / WH;
  const int k = meta_k(m.z);
  const int gh = ((class_first_sample(V, cls, V.Q) + k * V.Q) % V.nb) / V.Q;
  const int n = class_samples(V, cls, V.Q), hs = V.hs;
  const int j = hs > 1 ? range_of(k, n, hs) : 0;
  const bool more = k + 1 < (hs > 1 ? range_begin(j + 1, n, hs) : n);
  const size_t Ps = (size_t)p.P;
  float* rec = hs > 1 ? P.hsub + (size_t)(V.hbase + m.y) * 64 : nullptr;
  // the hero member's sample total (the companions' terms went straight into
  // their range sums as they were measured); nothing to add leaves the sums
  // untouched until the range ends (a Kahan step with a zero term would only
  // move compensation into the sum)
  const float4 v = P.part[slot];
  const bool zero = v.x == 0.0f && (NS == 1 || (v.y == 0.0f && v.z == 0.0f && v.w == 0.0f));
  float4 sh = make_float4(0.0f, 0.0f, 0.0f, 0.0f), ch = sh;
  if (!more || !zero) {
    sh = P.haccS[gh * Ps + slot];
    ch = P.haccC[gh * Ps + slot];
    kahan_add(sh.x, ch.x, v.x);
    if (NS == 4) {
      kahan_add(sh.y, ch.y, v.y);
      kahan_add(sh.z, ch.z, v.z);
      kahan_add(sh.w, ch.w, v.w);
    }
    if (more) {
      P.haccS[gh * Ps + slot] = sh;
      P.haccC[gh * Ps + slot] = ch;
    }
  }
  if (!more) {
    for (int g = 0; g < 4; ++g) {
      const float4 sm = g == gh ? sh : P.haccS[g * Ps + slot], c = g == gh ? ch : P.haccC[g * Ps + slot];
      if (hs > 1) {
        *(float4*)(rec + j * 16 + g * 4) = make_float4(sm.x - c.x, sm.y - c.y, sm.z - c.z, sm.w - c.w);
      } else {
        const size_t idx = ((size_t)m.y + (size_t)g * V.Q * WH) * NS;
        const float tot[4] = {sm.x - c.x, sm.y - c.y, sm.z - c.z, sm.w - c.w};
        for (int q = 0; q < NS; ++q) {
          float a = V.acc_sum[idx + q], e = V.acc_comp[idx + q];
          kahan_add(a, e, tot[q]);
          V.acc_sum[idx + q] = a;
          V.acc_comp[idx + q] = e;
        }
      }
    }
  }
  if (!more && hs > 1) {
    // publish this range's totals, then count it; the last range reads the
    // others' from L2
    __threadfence();
    if (atomicAdd(P.hsub_n + V.hbase + m.y, 1) == hs - 1) {
      __threadfence();
      for (int g = 0; g < 4; ++g) {
        const size_t idx = ((size_t)m.y + (size_t)g * V.Q * WH) * NS;
        for (int q = 0; q < NS; ++q) {
          float a = V.acc_sum[idx + q], e = V.acc_comp[idx + q];
          for (int r = 0; r < hs; ++r) kahan_add(a, e, __ldcg(rec + r * 16 + g * 4 + q));
          V.acc_sum[idx + q] = a;
          V.acc_comp[idx + q] = e;
        }
      }
    }
  }
  return more;
}

template <int NS, bool HERO>
__global__ void __launch_bounds__(256) k_regen(RenderParams p) {
  const Pool& P = p.pool;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    p.ctr->dq_count = 0;
    p.ctr->iters += 1;
  }
  int finished = 0, held = 0;
  // regeneration threshold: new tickets are claimed only while enough of the
  // pool was idle after the previous iteration (or when nothing is active)
  const int active_prev = *(volatile int*)&p.ctr->last_active;
  // the render is complete (no slot was live in the previous iteration and no
  // ticket is left): nothing to fold, claim or queue -- the iterations the
  // host loop runs past the end (it reads the counters a batch late) cost a
  // launch, not a scan of every slot
  // (decided once per block: other blocks' claims move next_ticket meanwhile)
  __shared__ int s_complete;
  if (threadIdx.x == 0)
    s_complete = active_prev == 0 && *(volatile unsigned long long*)&p.ctr->next_ticket >= p.ctr->total_tickets;
  __syncthreads();
  if (s_complete) return;
  const bool may_claim = p.regen_thr <= 0 || active_prev == 0 ||
                         (long long)(p.P - active_prev) * 100 >= (long long)p.regen_thr * p.P;
  // the views' first tickets, for the claims' view search (batches of views)
  __shared__ long long s_base[GR_REGEN_SMEM_VIEWS];
  const bool staged = p.n_views > 1 && p.n_views <= GR_REGEN_SMEM_VIEWS;
  if (staged) {
    for (int i = threadIdx.x; i < p.n_views; i += blockDim.x) s_base[i] = p.views[i].ticket_base;
    __syncthreads();
  }
  // each thread takes GR_REGEN_SLOTS slots per round (coalesced: slot j of a
  // round is base + j * blockDim.x + threadIdx.x), so the block's ticket
  // claims and queue reservations cost one barrier round and one atomic per
  // GR_REGEN_SLOTS slots
  constexpr int R = GR_REGEN_SLOTS;
  const int chunk = blockDim.x * R;
  for (int base = blockIdx.x * chunk; base < p.P; base += gridDim.x * chunk) {
    unsigned need_m = 0u, active_m = 0u, fresh_m = 0u, busy_m = 0u;  // per slot j: bit j
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
      const int slot = base + j * blockDim.x + threadIdx.x;
      if (slot >= p.P) break;
      bool need = false, active = false, fresh = false;
      // one byte of state per slot; the meta record only for finished samples
      const int st = P.st8[slot];
      const int4 m = st == ST_DONE ? P.meta[slot] : make_int4(0, 0, 0, 0);
      if (st == ST_DONE && HERO) {
        ++finished;
        if (fold_class<NS>(p, slot, m)) {
          start_sample<NS, true>(p, slot, m.x, m.y, meta_k(m.z) + 1);
          active = fresh = true;
        } else {
          need = true;
        }
      } else if (st == ST_DONE) {
        ++finished;
        const DevView& V = p.views[m.x];
        const int WH = V.W * V.H;
        const int bin = m.y / WH;
        const int k = meta_k(m.z) + 1;
        const int n_smp = bin_samples(V, bin);
        // a one-sample ticket's sum is its sample: no slot accumulator is kept
        // (the same bits as a Kahan sum of one term)
        float4 s = n_smp == 1 ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : P.accS[slot];
        float4 c = n_smp == 1 ? make_float4(0.0f, 0.0f, 0.0f, 0.0f) : P.accC[slot];
        const float4 v = P.part[slot];
        kahan_add(s.x, c.x, v.x);
        if (NS == 4) {
          kahan_add(s.y, c.y, v.y);
          kahan_add(s.z, c.z, v.z);
          kahan_add(s.w, c.w, v.w);
        }
        if (k < n_smp) {
          P.accS[slot] = s;
          P.accC[slot] = c;
          start_sample<NS, false>(p, slot, m.x, m.y, k);
          active = fresh = true;
        } else {
          // ticket complete: add its sum into the frame accumulator (Kahan)
          const size_t idx = (size_t)m.y * NS;
          float tot[4] = {s.x - c.x, s.y - c.y, s.z - c.z, s.w - c.w};
          for (int q = 0; q < NS; ++q) {
            float a = V.acc_sum[idx + q], e = V.acc_comp[idx + q];
            kahan_add(a, e, tot[q]);
            V.acc_sum[idx + q] = a;
            V.acc_comp[idx + q] = e;
          }
          need = true;
        }
      } else if (st == ST_IDLE) {
        need = true;
      } else if (st == ST_ACTIVE) {
        active = true;
      } else if (st == ST_WAIT) {
        // the sample's next-event ray is traced and measured in this
        // iteration: it is folded by the next regen pass
        P.st8[slot] = ST_DONE;
        ++held;
      }
      if (need && !may_claim) {
        need = false;
        if (st != ST_IDLE) P.st8[slot] = ST_IDLE;
      }
      need_m |= (unsigned)need << j;
      active_m |= (unsigned)active << j;
      fresh_m |= (unsigned)fresh << j;
      busy_m |= (unsigned)(st != ST_IDLE) << j;
    }
    // claim tickets, one atomic per block per pass (tickets without samples
    // in this render are skipped by claiming again)
    while (__syncthreads_or(need_m != 0u)) {
      const unsigned long long t0 = block_reserve_n<unsigned long long>(&p.ctr->next_ticket, __popc(need_m));
      unsigned long long t = t0;
#pragma unroll 1
      for (int j = 0; j < R; ++j) {
        if (!((need_m >> j) & 1u)) continue;
        const int slot = base + j * blockDim.x + threadIdx.x;
        const unsigned long long tk = t++;
        if (tk >= p.ctr->total_tickets) {
          need_m &= ~(1u << j);
          if ((busy_m >> j) & 1u) P.st8[slot] = ST_IDLE;
          continue;
        }
        int view = find_view(p, tk, staged ? s_base : nullptr);
        const DevView& V = p.views[view];
        // tickets run pixel-major, sample class fastest: neighbouring
        // slots start the same pixel at neighbouring wavelengths, so a warp's
        // camera rays (and grating orders) stay coherent.  Only classes that
        // receive samples have tickets: sample s goes to class s mod Q, so
        // with spp < Q they are the nbu = spp classes from first_sample mod Q
        // on.  The ticket's element is class * W*H + pixel, whatever the
        // claim order (with Q = nb the class is the bin).
        // (with hero-wavelength MIS and hs > 1, the class's sample ranges
        // come next: ticket = (pixel * hs + range) * nbu + class offset)
        const int local = (int)(tk - (unsigned long long)V.ticket_base);
        const int t = local / V.nbu;
        const int cls = (V.first_sample + (local - t * V.nbu)) % V.Q;
        const int pix = HERO ? t / V.hs : t;
        const int rng_j = HERO ? t - pix * V.hs : 0;
        if (class_samples(V, cls, V.Q) > 0) {
          if (HERO) {
            for (int g = 0; g < 4; ++g) {
              P.haccS[(size_t)g * p.P + slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
              P.haccC[(size_t)g * p.P + slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            }
          } else if (class_samples(V, cls, V.Q) > 1) {
            P.accS[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            P.accC[slot] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
          }
          const int k0 = HERO && V.hs > 1 ? range_begin(rng_j, class_samples(V, cls, V.Q), V.hs) : 0;
          start_sample<NS, HERO>(p, slot, view, cls * (V.W * V.H) + pix, k0);
          active_m |= 1u << j;
          fresh_m |= 1u << j;
          need_m &= ~(1u << j);
        }
      }
    }
    // compact live slots into the trace queue, one atomic per block per
    // part: continuing segments (incoherent, longer traversals) from the front
    // of the array, camera rays from the back, so that the queue is traced
    // longest-first and the end of the trace launch waits on short rays
    const unsigned cont_m = active_m & ~fresh_m;
    int qf = block_reserve_n<int>(&p.ctr->tq_count, __popc(cont_m));
    int qb = block_reserve_n<int>(&p.ctr->tq_back, __popc(fresh_m));
#pragma unroll 1
    for (int j = 0; j < R; ++j) {
      const int slot = base + j * blockDim.x + threadIdx.x;
      if ((fresh_m >> j) & 1u)
        P.tq[p.P - 1 - qb++] = slot;
      else if ((cont_m >> j) & 1u)
        P.tq[qf++] = slot;
    }
  }
  block_count(&p.ctr->samples, finished);
  block_count(&p.ctr->held, held);
}

// ------------------------------------------------------------------ trace
#ifndef GR_TRACE_REFILL
#define GR_TRACE_REFILL 12
#endif
#ifndef GR_LEAF_BATCH
#define GR_LEAF_BATCH 16
#endif
// queue entries a warp claims with one atomic: 32, or 64 for launches of
// more than GR_TRACE_BIG_QUEUE rays, where the atomics on the shared cursor
// add up and the end-of-launch imbalance of larger groups does not
#ifndef GR_TRACE_BIG_QUEUE
#define GR_TRACE_BIG_QUEUE (1 << 22)
#endif
#ifndef GR_LEAF_BLOCKED
#define GR_LEAF_BLOCKED 8
#endif
// node visits a lane makes between two looks at the warp's schedule
#ifndef GR_TRACE_STEPS
#define GR_TRACE_STEPS 6
#endif
// Closest hits for a queue of rays on the binary tree, one warp keeping its 32
// lanes busy across rays.  Warps claim the queue in groups of 32 entries from
// `cursor`; a lane whose ray has finished stays idle until GR_TRACE_REFILL
// lanes are idle (or every lane is), then the idle lanes take the next
// entries together, so ray set-up runs once per batch rather than once per
// lane, the warp no longer waits for the slowest ray of a fixed group of 32,
// and all warps advance through the queue together (neighbouring rays share
// BVH nodes in L1).  Leaf triangles are queued per lane (up to 3; a lane
// holding 2 stops walking) and tested in warp-wide passes once GR_LEAF_BATCH
// lanes hold some, or GR_LEAF_BLOCKED lanes are stopped, or no lane can walk:
// one test then serves many lanes instead of two or three.  The hit equals
// closest_hit's (the least (t, id) over the triangles whose boxes the ray
// enters); only the counts of visits and tests differ.
//   entry(e) -> slot of queue entry e; ray(slot, o, d, exclude) gives the
//   ray and returns its scene; done(slot, hit) consumes a finished ray.
template <bool HALF, class Entry, class Ray, class Done>
__device__ __forceinline__ void lane_trace(const RenderParams& p, int n, int* cursor, Entry&& entry, Ray&& ray,
                                           Done&& done, int& refined, int& visits, int& tests, int& err) {
  const int lane = threadIdx.x & 31;
  const unsigned below = (1u << lane) - 1u;
  BinTrav s;
  s.t = 0.0f;
  s.slot = -1;
  int stack[kStackDepth];
  const void* nodes = nullptr;
  const float4* tri = nullptr;
  int out = -1;
  bool live = false;     // the lane holds a ray
  bool walking = false;  // ... whose node walk has not ended
  int np = 0, pl0 = 0, pl1 = 0, pl2 = 0;  // queued leaves (at most 3)
  int exclude = -1;                        // the ray's s.exclude, kept for the queueing test
  auto queue_leaf = [&](int leaf) {
    if (leaf == exclude) return;
    if (np == 0) pl0 = leaf;
    else if (np == 1) pl1 = leaf;
    else pl2 = leaf;
    ++np;
  };
  auto finish = [&]() {
    Hit h;
    h.t = s.t;
    h.slot = s.slot;
    done(out, h);
    live = false;
  };
  // the warp's claimed group: its last `left` entries (from base + group - left) are unread
  const int group = n > GR_TRACE_BIG_QUEUE ? 64 : 32;
  int base = 0, left = 0;
  bool more = true;  // unclaimed groups may remain
  for (;;) {
    const unsigned idle = __ballot_sync(0xffffffffu, !live);
    if (idle == 0xffffffffu && !more && left == 0) break;
    const int nidle = __popc(idle);
    if ((left > 0 || more) && (nidle >= GR_TRACE_REFILL || idle == 0xffffffffu)) {
      const int rank = __popc(idle & below);
      int take = rank < left ? base + group - left + rank : -1;
      if (nidle <= left) {
        left -= nidle;
      } else {
        const int from_old = left;
        left = 0;
        if (more) {
          int nb = 0;
          if (lane == 0) nb = atomicAdd(cursor, group);
          nb = __shfl_sync(0xffffffffu, nb, 0);
          if (nb >= n) {
            more = false;
          } else {
            if (rank >= from_old) take = nb + (rank - from_old);
            base = nb;
            left = group - (nidle - from_old);
          }
        }
      }
      if (!live && take >= 0 && take < n) {
        const int slot = entry(take);
        int x = -1;
        float3 o, d;
        const DevScene& S = ray(slot, o, d, x);
        nodes = HALF ? (const void*)S.hnodes : (const void*)S.nodes;
        tri = S.tri;
        out = slot;
        np = 0;
        exclude = x;
        live = walking = !bin_begin(S.n_tris, tri, s, o, d, x, &refined, &tests);
        if (!live) {
          live = true;
          finish();
        }
      }
    }
    // leaf pass: the queued triangles of many lanes are tested together
    const bool blocked = live && (np >= 2 || (!walking && np > 0));
    const unsigned pend = __ballot_sync(0xffffffffu, live && np > 0);
    const unsigned blk = __ballot_sync(0xffffffffu, blocked);
    const unsigned can_walk = __ballot_sync(0xffffffffu, live && walking && np < 2);
    if (pend && (__popc(pend) >= GR_LEAF_BATCH || __popc(blk) >= GR_LEAF_BLOCKED || can_walk == 0)) {
      if (live && np > 0) {
        bin_leaf(tri, s, pl0, &refined, &tests);
        if (np > 1) bin_leaf(tri, s, pl1, &refined, &tests);
        if (np > 2) bin_leaf(tri, s, pl2, &refined, &tests);
        np = 0;
        if (!walking) finish();
      }
    }
#pragma unroll 1
    for (int k = 0; k < GR_TRACE_STEPS && live && walking && np < 2; ++k) {
      walking = !bin_step<HALF>(nodes, s, stack, &visits, &err, queue_leaf);
      if (!walking && np == 0) finish();
    }
  }
}

// Closest hits of the trace queue and of the next-event rays the previous
// k_shade requested, in one launch: the binary tree (FP32 or FP16 child boxes)
// through lane_trace, the 4-wide tree one ray per thread per pass.  Entries
// [0, ns) are the next-event rays (origin: the vertex, direction: the sampled
// emitter direction; their hits go to shh), then the trace queue, which holds
// continuing segments from the front of its array and camera rays from the
// back.  The few next-event rays ride on the launch's load balancing instead
// of a launch of their own, where the slowest of them set its length.
__device__ __forceinline__ int trace_entry(const RenderParams& p, int e, int ns, int front) {
  return e < ns ? (p.pool.sq[e] | kShadowEntry) : tq_entry(p, e - ns, front);
}

template <int TREE>
__global__ void __launch_bounds__(TREE == kTreeWide ? 256 : GR_TRACE_BLOCK, TREE == kTreeWide ? 3 : GR_TRACE_MIN_BLOCKS)
    k_trace(RenderParams p) {
  const Pool& P = p.pool;
  const int front = *(volatile int*)&p.ctr->tq_count;
  const int nt = front + *(volatile int*)&p.ctr->tq_back;
  const int ns = *(volatile int*)&p.ctr->sq_count;
  const int n = ns + nt;
  if (blockIdx.x == 0 && threadIdx.x == 0) p.ctr->segments += (unsigned long long)nt;
  int err = 0, refined = 0, visits = 0, tests = 0;
  if (TREE == kTreeWide) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const int es = trace_entry(p, i, ns, front);
      const int slot = es & ~kShadowEntry;
      const int4 m = P.meta[slot];
      const DevView& V = p.views[m.x];
      const DevScene& S = p.scenes[V.scene_index];
      const float4 a = P.od0[slot], b = (es & kShadowEntry) ? P.shd[slot] : P.od1[slot];
      const Hit h = closest_hit_wide(S, xyz(a), xyz(b), m.w, &refined, &visits, &tests, &err);
      (es & kShadowEntry ? P.shh : P.hit)[slot] = make_float2(h.t, __int_as_float(h.slot));
    }
  } else {
    lane_trace<TREE == kTreeHalf>(
        p, n, &p.ctr->trace_next, [&](int e) { return trace_entry(p, e, ns, front); },
        [&](int es, float3& o, float3& d, int& exclude) -> const DevScene& {
          const int slot = es & ~kShadowEntry;
          int4 m;
          float4 a, b;
          if (es & kShadowEntry) {
            // read again by k_shadow and k_shade: cached loads
            m = P.meta[slot];
            a = P.od0[slot];
            b = P.shd[slot];
          } else {
            // the slot state is read once per segment: evict-first loads
            // keep it from displacing the BVH and triangles in L2
            m = __ldcs(&P.meta[slot]);
            a = __ldcs(&P.od0[slot]);
            b = __ldcs(&P.od1[slot]);
          }
          o = xyz(a);
          d = xyz(b);
          exclude = m.w;
          return p.scenes[p.views[m.x].scene_index];
        },
        [&](int es, const Hit& h) {
          const float2 r = make_float2(h.t, __int_as_float(h.slot));
          if (es & kShadowEntry)
            P.shh[es & ~kShadowEntry] = r;
          else
            __stcs(&P.hit[es], r);
        },
        refined, visits, tests, err);
  }
  block_count(&p.ctr->ref_hit, refined);
  block_count(&p.ctr->node_visits, visits);
  block_count(&p.ctr->tri_tests, tests);
  if (err) atomicOr(&p.ctr->err, err);
}

// ------------------------------------------------------------------ footprint
// Free-space update of the footprint after a segment of t metres at
// wavenumber kw = 2 pi / lambda (1/um), Eq. K_free_space_propagation with
// zbar = z / |k|, z in um:
//   beta^2 <- beta^2 + 2 zbar rho + zbar^2 (1 + rho^2) / beta^2
//   rho    <- rho + zbar (1 + rho^2) / beta^2
__device__ __forceinline__ void footprint_update(float t_m, float kw, float& beta2, float& rho) {
  const float zbar = t_m * 1e6f / kw;
  const float b2 = beta2 + 2.0f * zbar * rho + zbar * zbar * (1.0f + rho * rho) / beta2;
  const float ro = rho + zbar * (1.0f + rho * rho) / beta2;
  beta2 = b2;
  rho = ro;
}
// The same update given 1/|k| (um), with one reciprocal instead of divisions
// (the class wavelengths of hero-wavelength MIS).
__device__ __forceinline__ void footprint_update_ik(float t_m, float ik, float& beta2, float& rho) {
  const float zbar = t_m * 1e6f * ik;
  const float f = zbar * (1.0f + rho * rho) * __frcp_rn(beta2);
  const float b2 = beta2 + 2.0f * zbar * rho + zbar * f;
  rho = rho + f;
  beta2 = b2;
}

// The path's footprint at a class wavelength of hero-wavelength MIS, from the
// hero's: interactions leave (beta, rho) unchanged (Eq.
// K_reflection_refraction, Eq. K_grating) and a free segment adds zbar = z /
// |k| to the footprint's complex parameter (Eq. K_free_space_propagation
// composes additively: rho grows by zbar / Kr with Kr = beta^2 / (1 + rho^2)
// fixed), so from the camera's (beta0^2, 0), the same at every wavelength,
// rho = Zbar / beta0^2 and beta^2 = beta0^2 (1 + rho^2), where Zbar, the sum
// of the path's zbar, scales with the wavelength (every member's segments use
// the hero's medium index; a dispersive medium drops the companions).
// ratio = lambda_g / lambda_hero.
__device__ __forceinline__ void member_footprint(float rho_hero, float ratio, float beta02, float& beta2, float& rho) {
  rho = rho_hero * ratio;
  beta2 = beta02 * (1.0f + rho * rho);
}

// ------------------------------------------------------------------ measurement
// Emitter measurement (Eq. measurement_operator on an emissive triangle set):
// one footprint point x ~ N(0, beta^2/2) transverse to d, projected along d
// onto the emitter plane and tested for coverage; the local mean direction is
// shifted by rho x / (beta^2 |k|) with residual angular variance
// 1/(2 beta^2 |k|^2); the source emits a Gaussian lobe of spread lambda/lc
// about its normal.  The lobe's quadratic form is evaluated in FP64.
// Coverage of the footprint point pt (m), projected along d onto the plane
// (normal ne, through v0) of emitter E: inside any of its triangles
// (barycentric test, edges inclusive).
__device__ __forceinline__ bool emitter_covers(const DevScene& S, const DevEmitter& E, float3 pt, float3 d, float3 ne,
                                               float3 v0p) {
  const float tp = dot(v0p - pt, ne) / dot(d, ne);
  const float3 q = pt + tp * d;
  bool covered = false;
  for (int i = 0; i < E.count && !covered; ++i) {
    const float3 v0 = xyz(S.emitter_tris[3 * (E.first + i)]);
    const float3 a = xyz(S.emitter_tris[3 * (E.first + i) + 1]) - v0;
    const float3 b = xyz(S.emitter_tris[3 * (E.first + i) + 2]) - v0;
    const float3 c = q - v0;
    const float daa = dot(a, a), dab = dot(a, b), dbb = dot(b, b), dca = dot(c, a), dcb = dot(c, b);
    const float den = daa * dbb - dab * dab;
    const float bu = (dbb * dca - dab * dcb) / den;
    const float bv = (daa * dcb - dab * dca) / den;
    covered = bu >= 0.0f && bv >= 0.0f && bu + bv <= 1.0f;
  }
  return covered;
}

__device__ float measure_emitter(const DevScene& S, int ei, float3 hit, float3 d, float beta2, float rho, float k,
                                 float lambda, float u0, float u1) {
  const DevEmitter E = S.emitters[ei];
  const gr_material& M = S.mats[E.mat];
  const float4 t0 = S.emitter_tris[3 * E.first];
  const d3 ned = d3{E.nd[0], E.nd[1], E.nd[2]};  // normal computed once per scene
  const float3 ne = f3(E.n[0], E.n[1], E.n[2]);
  if (dot(d, ne) >= 0.0f) return 0.0f;
  float z0, z1;
  box_muller(u0, u1, z0, z1);
  const float sigma = sqrtf(0.5f * beta2);
  float3 e1, e2;
  onb(d, e1, e2);
  const float3 x_um = (sigma * z0) * e1 + (sigma * z1) * e2;
  if (!emitter_covers(S, E, hit + 1e-6f * x_um, d, ne, xyz(t0))) return 0.0f;
  const float3 mu = (rho / (beta2 * k)) * x_um;
  // FP64 quadratic form of the measured lobe
  const d3 dl = dnormalize(dadd(D3(d), D3(mu)));
  const d3 w = d3{-dl.x, -dl.y, -dl.z};
  const d3 diff = dsub(w, ned);
  const double sc2 = 1.0 / (2.0 * (double)beta2 * (double)k * (double)k);
  double s2 = 0.0;
  if (M.coh_len_um > 0.0f) {
    double s = (double)lambda / (double)M.coh_len_um;
    s2 = s * s;
  }
  const double kappa = 1.0 / (sc2 + s2);
  const double q2 = 0.5 * kappa * ddot(diff, diff);
  const float kf = (float)kappa;
  const float pref = kf < 1e-8f ? 0.25f / kPi : kf / (2.0f * kPi * (-expm1f(-2.0f * kf)));
  return M.Le * pref * expf(-(float)q2);
}

// ------------------------------------------------------------------ anisotropic footprints
// Anisotropic generalized rays (GR_FLAG_ANISO; beta and rho as matrices,
// Sec. 3.1 and Eq. def_gen_ray, with the general form derived from the
// Gaussian field): the transverse field exp(-x^T A x / 2) is kept as K = A^-1
// = Kr + i Ki (um^2) in the ray's frame (f, d x f).  Free propagation adds
// i zbar I; an interaction maps K by the surface's anamorphic map W = P_out
// P_in^-1 (P: a tangent basis projected onto the transverse frames).  With
// S = (Kr + Ki Kr^-1 Ki) / 2 the spatial covariance, a footprint point x has
// direction shift Kr^-1 Ki S^-1 x / (2|k|) and residual angular covariance
// S^-1 / (4|k|^2); the wavevector marginal is Kr^-1 / 2.  Only Kr, which
// propagation leaves unchanged, is inverted, so FP32 does not cancel.
struct AK {
  float r11, r12, r22, i11, i12, i22;
};
__device__ __forceinline__ void sym_inv(float a, float b, float c, float& ia, float& ib, float& ic) {
  const float id = 1.0f / (a * c - b * b);
  ia = c * id;
  ib = -b * id;
  ic = a * id;
}
// W K W^T (real W)
__device__ __forceinline__ AK ak_congruence(const float W[2][2], const AK& K) {
  AK r;
  r.r11 = W[0][0] * W[0][0] * K.r11 + 2.0f * W[0][0] * W[0][1] * K.r12 + W[0][1] * W[0][1] * K.r22;
  r.r12 = W[0][0] * W[1][0] * K.r11 + (W[0][0] * W[1][1] + W[0][1] * W[1][0]) * K.r12 + W[0][1] * W[1][1] * K.r22;
  r.r22 = W[1][0] * W[1][0] * K.r11 + 2.0f * W[1][0] * W[1][1] * K.r12 + W[1][1] * W[1][1] * K.r22;
  r.i11 = W[0][0] * W[0][0] * K.i11 + 2.0f * W[0][0] * W[0][1] * K.i12 + W[0][1] * W[0][1] * K.i22;
  r.i12 = W[0][0] * W[1][0] * K.i11 + (W[0][0] * W[1][1] + W[0][1] * W[1][0]) * K.i12 + W[0][1] * W[1][1] * K.i22;
  r.i22 = W[1][0] * W[1][0] * K.i11 + 2.0f * W[1][0] * W[1][1] * K.i12 + W[1][1] * W[1][1] * K.i22;
  return r;
}
// K across an interaction at normal n: (f_in, d_in) -> (f_out, d_out)
__device__ AK ak_interaction(const AK& K, float3 f_in, float3 d_in, float3 f_out, float3 d_out, float3 n) {
  float3 s1, s2;
  onb(n, s1, s2);
  const float3 u2 = cross(d_in, f_in), v2 = cross(d_out, f_out);
  const float p00 = dot(f_in, s1), p01 = dot(f_in, s2), p10 = dot(u2, s1), p11 = dot(u2, s2);
  const float q00 = dot(f_out, s1), q01 = dot(f_out, s2), q10 = dot(v2, s1), q11 = dot(v2, s2);
  const float id = 1.0f / (p00 * p11 - p01 * p10);
  const float i00 = p11 * id, i01 = -p01 * id, i10 = -p10 * id, i11 = p00 * id;
  const float W[2][2] = {{q00 * i00 + q01 * i10, q00 * i01 + q01 * i11}, {q10 * i00 + q11 * i10, q10 * i01 + q11 * i11}};
  return ak_congruence(W, K);
}
// An angular lobe of 2D precision (c11, c12, c22) in the frame (f1, f2),
// written so that an isotropic precision kappa I is the vMF exactly: kbar
// |dv|^2 / 2 (kbar = the mean of the eigenvalues) plus the traceless part on
// the transverse components, normalised with the vMF constant of
// kappa_eff = sqrt(det); |dv|^2 is taken in FP64 by the caller where the
// lobe can be narrow.
__device__ __forceinline__ float aniso_lobe_q(double dv2, float t1, float t2, float c11, float c12, float c22) {
  const float kbar = 0.5f * (c11 + c22);
  return 0.5f * (float)((double)kbar * dv2) + 0.5f * ((c11 - kbar) * t1 * t1 + 2.0f * c12 * t1 * t2 + (c22 - kbar) * t2 * t2);
}
__device__ __forceinline__ float aniso_lobe_pref(float c11, float c12, float c22) {
  const float ke = sqrtf(fmaxf(0.0f, c11 * c22 - c12 * c12));
  return ke < 1e-8f ? 0.25f / kPi : ke / (2.0f * kPi * (-expm1f(-2.0f * ke)));
}
// Distant source seen by an anisotropic ray: wavevector marginal Kr^-1 / 2
// (over |k|^2) plus the source's spread.
__device__ float measure_distant_aniso(const gr_light& L, float3 d, float lambda, float k, const AK& K, float3 xf) {
  if (L.type == GR_LIGHT_ENV) return L.E;
  float a, b, c;
  sym_inv(K.r11, K.r12, K.r22, a, b, c);
  const float s2 = src_spread2(lambda, L.coh_len_um), ik2 = 0.5f / (k * k);
  float c11, c12, c22;
  sym_inv(a * ik2 + s2, b * ik2, c * ik2 + s2, c11, c12, c22);
  const float3 dv = d - f3(L.dir[0], L.dir[1], L.dir[2]);
  const float q = aniso_lobe_q((double)dot(dv, dv), dot(dv, xf), dot(dv, cross(d, xf)), c11, c12, c22);
  return L.E * aniso_lobe_pref(c11, c12, c22) * expf(-q);
}

// Emitter seen by an anisotropic ray: the footprint point from the spatial
// covariance S (Cholesky factor in the frame onb(d)), its direction shift and
// residual lobe, the lobe's isotropic part in FP64 as in measure_emitter.
__device__ float measure_emitter_aniso(const DevScene& S, int ei, float3 hit, float3 d, const AK& K, float3 xf,
                                       float k, float lambda, float u0, float u1) {
  const DevEmitter E = S.emitters[ei];
  const gr_material& M = S.mats[E.mat];
  const float4 t0 = S.emitter_tris[3 * E.first];
  const d3 ned = d3{E.nd[0], E.nd[1], E.nd[2]};
  const float3 ne = f3(E.n[0], E.n[1], E.n[2]);
  if (dot(d, ne) >= 0.0f) return 0.0f;
  float z0, z1;
  box_muller(u0, u1, z0, z1);
  float3 e1, e2;
  onb(d, e1, e2);
  const float3 u2 = cross(d, xf);
  const float R[2][2] = {{dot(e1, xf), dot(e1, u2)}, {dot(e2, xf), dot(e2, u2)}};
  const AK Ke = ak_congruence(R, K);
  // S = (Kr + Ki Kr^-1 Ki) / 2
  float a, b, c;
  sym_inv(Ke.r11, Ke.r12, Ke.r22, a, b, c);
  const float m11 = Ke.i11 * a + Ke.i12 * b, m12 = Ke.i11 * b + Ke.i12 * c;  // Ki Kr^-1
  const float m21 = Ke.i12 * a + Ke.i22 * b, m22 = Ke.i12 * b + Ke.i22 * c;
  const float s11 = 0.5f * (Ke.r11 + m11 * Ke.i11 + m12 * Ke.i12);
  const float s12 = 0.5f * (Ke.r12 + m11 * Ke.i12 + m12 * Ke.i22);
  const float s22 = 0.5f * (Ke.r22 + m21 * Ke.i12 + m22 * Ke.i22);
  const float l11 = sqrtf(s11), l21 = s12 / l11, l22 = sqrtf(fmaxf(0.0f, s22 - l21 * l21));
  const float x1 = l11 * z0, x2 = l21 * z0 + l22 * z1;  // um
  if (!emitter_covers(S, E, hit + 1e-6f * (x1 * e1 + x2 * e2), d, ne, xyz(t0))) return 0.0f;
  // shift Kr^-1 Ki S^-1 x / (2k); residual covariance S^-1 / (4k^2) + spread
  float j11, j12, j22;
  sym_inv(s11, s12, s22, j11, j12, j22);
  const float y1 = j11 * x1 + j12 * x2, y2 = j12 * x1 + j22 * x2;
  const float v1 = Ke.i11 * y1 + Ke.i12 * y2, v2 = Ke.i12 * y1 + Ke.i22 * y2;
  const float hk = 0.5f / k;
  const float mu1 = hk * (a * v1 + b * v2), mu2 = hk * (b * v1 + c * v2);
  const float s2 = src_spread2(lambda, M.coh_len_um), q4 = 0.25f / (k * k);
  float c11, c12, c22;
  sym_inv(j11 * q4 + s2, j12 * q4, j22 * q4 + s2, c11, c12, c22);
  const d3 dl = dnormalize(dadd(D3(d), D3(mu1 * e1 + mu2 * e2)));
  const d3 diff = d3{-dl.x - ned.x, -dl.y - ned.y, -dl.z - ned.z};
  const float3 df = f3((float)diff.x, (float)diff.y, (float)diff.z);
  const float q = aniso_lobe_q(ddot(diff, diff), dot(df, e1), dot(df, e2), c11, c12, c22);
  return M.Le * aniso_lobe_pref(c11, c12, c22) * expf(-q);
}

// An emitter's unit normal (front face), computed in FP64 when the scene is
// created and stored rounded to FP32.
__device__ __forceinline__ float3 emitter_normal(const DevScene& S, int ei) {
  const DevEmitter& E = S.emitters[ei];
  return f3(E.n[0], E.n[1], E.n[2]);
}

// Density of the m >= 1 part of the rough lobe in tangential direction
// cosines at squared offset r2 from the mirror direction, kl2 = (|k| l)^2.
// Evaluated only where it is needed (MIS weights of paths that actually reach
// an emitter), not at every rough vertex.
// Term m of the sum is e^-g g^m / m! * kl2 / (4 pi m) * exp(-r2 kl2 / (4 m)):
// one reciprocal per term and no division; the sum stops once m has passed g
// and the Poisson weight is below 1e-13 (as rough_density_class).
__device__ float rough_density(float g, float kl2, float r2) {
  if (g > kGCont) {
    const float var = 2.0f * g / kl2;
    return __expf(-0.5f * r2 / var) / (2.0f * kPi * var);
  }
  const float c = 0.25f * r2 * kl2, a = kl2 * (0.25f / kPi);
  float pm = __expf(-g), sum = 0.0f;
  const int mmax = (int)(g + 12.0f * sqrtf(g) + 20.0f);
  for (int m = 1; m <= mmax; ++m) {
    const float inv = __frcp_rn((float)m);
    pm *= g * inv;
    sum += pm * (a * inv) * __expf(-c * inv);
    if ((float)m > g && pm < 1e-13f) break;
  }
  return sum;
}

// The same density at the four wavelengths of a hero class (roughness g_j,
// kl2_j = (|k_j| l)^2) at one squared offset r2, in one pass over the term
// count m: term m is e^-g g^m / m! * kl2 / (4 pi m) * exp(-r2 kl2 / (4 m)),
// one reciprocal per m shared by the four wavelengths and no division.  The
// sum stops once m has passed every g_j and every Poisson weight is below
// 1e-13 (or at rough_density's bound).  want[j] false gives 0.
__device__ void rough_density_class(const float g[4], const float kl2[4], const bool want[4], float r2, float out[4]) {
  float pm[4], c[4], a[4];
  bool pois[4];
  float gmax = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    out[j] = 0.0f;
    pois[j] = want[j] && g[j] > 0.0f && g[j] <= kGCont;
    if (want[j] && g[j] > kGCont) {
      const float var = 2.0f * g[j] / kl2[j];
      out[j] = __expf(-0.5f * r2 / var) / (2.0f * kPi * var);
    }
    pm[j] = pois[j] ? __expf(-g[j]) : 0.0f;
    c[j] = 0.25f * r2 * kl2[j];
    a[j] = kl2[j] * (0.25f / kPi);
    if (pois[j]) gmax = fmaxf(gmax, g[j]);
  }
  if (gmax == 0.0f) return;
  const int mmax = (int)(gmax + 12.0f * sqrtf(gmax) + 20.0f);
  for (int m = 1; m <= mmax; ++m) {
    const float inv = __frcp_rn((float)m);
    float big = 0.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      if (!pois[j]) continue;
      pm[j] *= g[j] * inv;
      out[j] += pm[j] * (a[j] * inv) * __expf(-c[j] * inv);
      big = fmaxf(big, pm[j]);
    }
    if ((float)m > gmax && big < 1e-13f) break;
  }
}

// Conservative precheck of a next-event ray toward emitter ei: false only if
// the ray's closest hit cannot be a front-face point of that (planar) emitter
// -- its plane is behind the ray or met from the back (where the emitter does
// not emit), or the ray meets the plane outside the emitter's bounding box
// widened by 1e-4 (1 + t) m, far above the FP32 error of the plane point.
// Near-grazing rays (|cos| < 1e-3) and non-planar emitters always pass.  A
// false result means a zero contribution, so the ray is not traced.
__device__ __forceinline__ bool emitter_reachable(const DevScene& S, int ei, float3 x, float3 w) {
  const DevEmitter E = S.emitters[ei];
  if (!E.planar) return true;
  const float3 ne = emitter_normal(S, ei);
  const float den = dot(w, ne);
  if (den >= 0.0f) return false;  // back face or parallel: measured as zero
  if (den > -1e-3f) return true;
  const float te = dot(xyz(S.emitter_tris[3 * E.first]) - x, ne) / den;
  if (!(te > 0.0f)) return false;
  const float3 q = x + te * w;
  const float m = 1e-4f * (1.0f + te);
  return q.x >= E.lo[0] - m && q.x <= E.hi[0] + m && q.y >= E.lo[1] - m && q.y <= E.hi[1] + m &&
         q.z >= E.lo[2] - m && q.z <= E.hi[2] + m;
}

// ------------------------------------------------------------------ shade
// Grating order pick from tabulated weights w_|j| = J_j(pi h / lambda)^2
// (Eq. K_grating): over the propagating orders (|t_mir + j lambda/Lambda g|^2
// < 1) the first j whose cumulative weight exceeds u * total (total = 1 when
// the weights are not renormalised), or 0x7fffffff if none does.
// `ambiguous` is set when the pick could differ from the one made with the
// exact weights, or no order is picked under renormalisation; the caller then
// re-decides at higher precision.  The window: each stored weight carries a
// relative error <= ut (plus an absolute <= at below the type's normal range),
// and n FP32 additions, the product u * total and the final subtraction each
// round by <= 2^-24 relative, so |(cum - target) - exact| <=
// (2 ut + 2 (n + 2) 2^-24) total + 2 n at; the window is 1.25 times that.
template <class Val>
__device__ __forceinline__ int grating_pick_tab(int jm, float3 t_mir, float step, float3 gt, bool renorm, float u,
                                                float ut, float at, Val val, bool& ambiguous) {
  float total = 0.0f;
  int n = 0;
  for (int j = -jm; j <= jm; ++j) {
    const float3 tj = t_mir + ((float)j * step) * gt;
    if (dot(tj, tj) < 1.0f) {
      total += val(j < 0 ? -j : j);
      ++n;
    }
  }
  const float tot_w = total;
  if (!renorm) total = 1.0f;
  const float target = u * total;
  float cum = 0.0f, prev = 0.0f;
  int pick = 0x7fffffff;
  for (int j = -jm; j <= jm; ++j) {
    const float3 tj = t_mir + ((float)j * step) * gt;
    if (dot(tj, tj) < 1.0f) {
      prev = cum;
      cum += val(j < 0 ? -j : j);
      if (cum > target) {
        pick = j;
        break;
      }
    }
  }
  const float eps = 1.25f * ((2.0f * ut + 2.0f * (float)(n + 2) * 5.9604645e-8f) * fmaxf(fmaxf(total, tot_w), 1e-30f) +
                             2.0f * (float)n * at);
  ambiguous = (pick != 0x7fffffff && (cum - target < eps || target - prev < eps)) || (pick == 0x7fffffff && renorm);
  return pick;
}

// Rounding of a stored order weight: relative bound (round to nearest in the
// type's normal range) and absolute bound below it.
template <typename TT>
struct TableRound;
template <>
struct TableRound<float> {
  static constexpr float rel = 5.9604645e-8f, abs = 1e-45f;  // 2^-24, subnormals
};
template <>
struct TableRound<__half> {
  static constexpr float rel = 4.8828125e-4f, abs = 2.9802322e-8f;  // 2^-11, 2^-25
};
template <>
struct TableRound<__nv_bfloat16> {
  static constexpr float rel = 3.90625e-3f, abs = 1e-38f;  // 2^-8, subnormals
};

// FP64 re-decisions, taken only when the FP32 pick lies within the tables'
// rounding of a CDF boundary; kept out of line so the rare path costs the
// common one neither code size nor registers.
//
// Grating order j (Eq. K_grating): cumulative J_j(pi h / lambda)^2 over the
// propagating orders (|t_mir + j lambda/Lambda g|^2 < 1), renormalised unless
// `renorm` is false; returns the first j whose cumulative sum exceeds
// u * total, or 0x7fffffff if none does.
__device__ __noinline__ int grating_pick_fp64(double lam_d, float height_um, int jm, float3 t_mir, float step,
                                              float3 gt, bool renorm, float u) {
  const double xarg = kPiD * (double)height_um / lam_d;
  double tot_d = 0.0;
  for (int j = -jm; j <= jm; ++j) {
    const float3 tj = t_mir + ((float)j * step) * gt;
    if (dot(tj, tj) < 1.0f) {
      const double J = bessel_j_d(j, xarg);
      tot_d += J * J;
    }
  }
  if (!renorm) tot_d = 1.0;
  const double tgt = (double)u * tot_d;
  double cd = 0.0;
  for (int j = -jm; j <= jm; ++j) {
    const float3 tj = t_mir + ((float)j * step) * gt;
    if (dot(tj, tj) < 1.0f) {
      const double J = bessel_j_d(j, xarg);
      cd += J * J;
      if (cd > tgt) return j;
    }
  }
  return 0x7fffffff;
}

// Rough-surface term count m ~ Poisson(g), g = (2 k sigma_h cos_i)^2: the
// first m whose cumulative Poisson probability exceeds u (at most 1000).
__device__ __noinline__ int poisson_pick_fp64(double lam_d, float sigma_h_um, float cos_i, float u) {
  const double kd = 2.0 * kPiD / lam_d;
  double gd = 2.0 * kd * (double)sigma_h_um * (double)cos_i;
  gd *= gd;
  double pd = exp(-gd), cd = pd;
  int mi = 0;
  while ((double)u >= cd && mi < 1000) {
    ++mi;
    pd *= gd / mi;
    cd += pd;
  }
  return mi;
}

// Probability of grating order 0 at one wavelength (Eq. K_grating): its
// weight J_0^2 over the total of the propagating orders (|t_mir + j step g|^2
// < 1), or the raw weight without renormalisation; from the FP32 copy of the
// order table.  Used for the density ratios of hero-wavelength MIS, where a
// probability (not a decision) is needed.
__device__ __forceinline__ float order0_prob(const TableRow& row, float3 t_mir, float step, float3 gt, bool renorm,
                                            const float* __restrict__ vals32) {
  const float a0 = __ldg(vals32 + row.offset);
  if (!renorm) return a0;
  float total = 0.0f;
  for (int j = -row.jmax; j <= row.jmax; ++j) {
    const float3 tj = t_mir + ((float)j * step) * gt;
    if (dot(tj, tj) < 1.0f) total += __ldg(vals32 + row.offset + (j < 0 ? -j : j));
  }
  return total > 0.0f ? a0 / total : 0.0f;
}

// An out-of-line copy of the emitter measurement for the hero-wavelength
// paths, which evaluate it once per class member: inlined four times over,
// the hero shading kernel outgrew the instruction cache (no-instruction
// stalls were 7.9 warps per issue in ncu); out of line, the kernel takes 50.1
// instead of 52.1 ms per headline step.  The plain paths keep the inlined
// form (out of line it cost them 0.25 ms).  Making the order-0 probability
// and the escape measurement out-of-line too gained nothing more.
__device__ __noinline__ float hero_measure_emitter(const DevScene& S, int ei, float3 hit, float3 d, float beta2,
                                                   float rho, float k, float lambda, float u0, float u1) {
  return measure_emitter(S, ei, hit, d, beta2, rho, k, lambda, u0, u1);
}
// Distant sources measured at class wavelength lg (escape, hero MIS).
__device__ __forceinline__ float hero_escape_measure(const DevScene& S, float3 d, float lg, float beta0) {
  const float kg = 2.0f * kPi * __frcp_rn(lg);
  const float s2g = 1.0f / (2.0f * beta0 * beta0 * kg * kg);
  float mg = 0.0f;
  for (int l = 0; l < S.n_lights; ++l) {
    const gr_light L = S.lights[l];
    if (L.type == GR_LIGHT_ENV) {
      mg += L.E;
    } else {
      const float kap = 1.0f / (s2g + src_spread2(lg, L.coh_len_um));
      mg += L.E * vmf(d, f3(L.dir[0], L.dir[1], L.dir[2]), kap);
    }
  }
  return mg;
}

// HERO: hero-wavelength spectral MIS (Sec. 7.2).  The path's bin is the hero
// of its class {c, c+Q, c+2Q, c+3Q} and makes every decision; hq[g] holds the
// path's density at class wavelength g divided by its density at the hero's
// (1 through wavelength-independent decisions, the ratio of order-0 or rough
// lobe densities, 0 after a dispersive delta); fb/fr carry the footprint at
// each class wavelength.  Every connection to a light is measured at each
// class wavelength: escapes (and emitter hits after a delta vertex) with the
// balance heuristic cf_g hq_g / sum_j cf_j hq_j (cf_j = the class's share of
// samples whose hero is bin j); emitter hits after a diffuse vertex and
// next-event estimates, with NEE on, with the power heuristic over the
// (wavelength, lobe or emitter sampling) pairs, which with one hero per class
// is the plain lobe/emitter power heuristic.
// MODE 0: plain; 1: hero-wavelength MIS (HERO); 2: anisotropic footprints
// (ANISO, K carried per slot).
template <int NS, typename TT, int MODE>
__global__ void __launch_bounds__(256, MODE == 1   ? GR_SHADE_MIN_BLOCKS_HERO
                                      : MODE == 2 ? GR_SHADE_MIN_BLOCKS_ANISO
                                                  : (NS == 1 ? GR_SHADE_MIN_BLOCKS_NS1 : GR_SHADE_MIN_BLOCKS))
    k_shade(RenderParams p) {
  constexpr bool HERO = MODE == 1, ANISO = MODE == 2;
  extern __shared__ __align__(16) unsigned char smem[];
  const TableRow* rows = p.rows;
  const TT* tvals = (const TT*)p.table_vals;
  if (p.table_smem) {
    TableRow* srows = (TableRow*)smem;
    TT* svals = (TT*)(smem + sizeof(TableRow) * p.table_rows);
    for (int i = threadIdx.x; i < p.table_rows; i += blockDim.x) srows[i] = p.rows[i];
    for (int i = threadIdx.x; i < p.table_vals_count; i += blockDim.x) svals[i] = ((const TT*)p.table_vals)[i];
    __syncthreads();
    rows = srows;
    tvals = svals;
  }
  const Pool& P = p.pool;
  // the iteration's trace queue, as k_shadow recorded it when it reset the
  // queue counters for the next regen pass
  const int front = *(volatile int*)&p.ctr->tq_front;
  const int n = *(volatile int*)&p.ctr->tq_n;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    bool want_shadow = false;
    bool want_density = false;  // hero: the class lobe densities are deferred to k_density
    int slot = -1;
    if (i < n) {
      slot = tq_entry(p, i, front);
      int4 m = P.meta[slot];
      const DevView& V = p.views[m.x];
      const DevScene& S = p.scenes[V.scene_index];
      float4 a0 = P.od0[slot], a1 = P.od1[slot];
      const float2 hh = P.hit[slot];
      float3 o = xyz(a0), d = xyz(a1);
      float beta2 = a0.w, rho = a1.w;
      const int kk = meta_k(m.z), seg = meta_seg(m.z), prev_delta = meta_delta(m.z);
      const int WH = V.W * V.H;
      const int cls = m.y / WH;  // the ticket's sample class (its bin without HERO)
      const int pixel = m.y - cls * WH;
      const int Qv = HERO ? V.Q : V.nb;
      const int smp = class_first_sample(V, cls, Qv) + kk * Qv;
      const int bin = HERO ? smp % V.nb : cls;
      const int gh = HERO ? (bin - cls) / Qv : 0;  // the hero's member of the class
      const float lambda = bin_lambda(V, bin);
      const float cstep = HERO ? bin_step(V) : 0.0f;
      const float kw = 2.0f * kPi / lambda;
      const float s_ray2 = 1.0f / (2.0f * V.beta0 * V.beta0 * kw * kw);
      float T[4][4];
      float4 xfv = make_float4(0.0f, 0.0f, 0.0f, 1.0f), pt;
      if (seg == 0) {
        // camera segment (nothing stored by start_sample): identity Mueller
        // matrix, no contribution yet, Stokes frame x axis = the camera's right
        // vector made orthogonal to d, medium air
        for (int r = 0; r < 4; ++r)
          for (int c = 0; c < 4; ++c) T[r][c] = r == c ? 1.0f : 0.0f;
        const float3 xf0 = NS == 1 && !ANISO ? f3(0.0f, 0.0f, 0.0f) : normalize(V.right - dot(V.right, d) * d);
        xfv = make_float4(xf0.x, xf0.y, xf0.z, 1.0f);
        pt = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      } else {
        if (NS == 1) {
          const float4 t0 = P.tp[0][slot];
          T[0][0] = t0.x;
          xfv.w = t0.y;  // the medium's index rides in the unused word of the scalar throughput
        } else {
          for (int r = 0; r < 4; ++r) {
            float4 v = P.tp[r][slot];
            T[r][0] = v.x;
            T[r][1] = v.y;
            T[r][2] = v.z;
            T[r][3] = v.w;
          }
        }
        if (NS == 4) xfv = P.xf[slot];
        if (NS == 1 && ANISO) {  // the footprint's frame
          const float4 f = P.xf[slot];
          xfv = make_float4(f.x, f.y, f.z, xfv.w);
        }
        pt = P.part[slot];
      }
      // anisotropic footprint: isotropic beta0^2 I on the camera segment
      AK K{beta2, 0.0f, beta2, 0.0f, 0.0f, 0.0f};
      if (ANISO && seg > 0) {
        const float4 k0 = P.ak0[slot], k1 = P.ak1[slot];
        K = AK{k0.x, k0.y, k0.z, k0.w, k1.x, k1.y};
      }
      float hq[4] = {1.0f, 1.0f, 1.0f, 1.0f};
      if (HERO && seg > 0) {
        const float4 q4 = P.hq[slot];
        hq[0] = q4.x;
        hq[1] = q4.y;
        hq[2] = q4.z;
        hq[3] = q4.w;
      }
      auto drop_companions = [&]() {
#pragma unroll
        for (int g = 0; g < 4; ++g)
          if (g != gh) hq[g] = 0.0f;
      };
      const int hslot = __float_as_int(hh.y);
      bool done = false;
      auto add_col = [&](float val) {
        pt.x += T[0][0] * val;
        if (NS == 4) {
          pt.y += T[1][0] * val;
          pt.z += T[2][0] * val;
          pt.w += T[3][0] * val;
        }
      };
      // a contribution to class member g: the hero's into the sample's own
      // sum, the others' straight into their range sums
      auto add_member = [&](int g, float val) {
        if (g == gh) {
          add_col(val);
          return;
        }
        member_add<NS>(P, (size_t)p.P, g, slot, T[0][0], NS == 4 ? T[1][0] : 0.0f, NS == 4 ? T[2][0] : 0.0f,
                       NS == 4 ? T[3][0] : 0.0f, val);
      };
      if (hslot < 0 && HERO) {
        // escape measured at every class wavelength, balance-heuristic weights
        float cf[4], den = 0.0f;
        class_shares(V, cls, Qv, cf);
#pragma unroll
        for (int g = 0; g < 4; ++g) den += cf[g] * hq[g];
#pragma unroll
        for (int g = 0; g < 4; ++g) {
          const float wq = cf[g] * hq[g];
          float val = 0.0f;
          if (wq > 0.0f) {
            const float mg = hero_escape_measure(S, d, step_lambda(V, cstep, cls + g * Qv), V.beta0);
            val = mg * (wq / den);
          }
          // a zero term leaves the member's sum as it is (the sums start at
          // +0 and a zero product cannot change them): no read-modify-write
          if (val != 0.0f) add_member(g, val);
        }
        done = true;
      } else if (hslot < 0 && ANISO) {
        float msum = 0.0f;
        for (int l = 0; l < S.n_lights; ++l) msum += measure_distant_aniso(S.lights[l], d, lambda, kw, K, xyz(xfv));
        add_col(msum);
        done = true;
      } else if (hslot < 0) {
        float msum = 0.0f;
        for (int l = 0; l < S.n_lights; ++l) {
          const gr_light L = S.lights[l];
          if (L.type == GR_LIGHT_ENV) {
            msum += L.E;
          } else {
            const float kap = 1.0f / (s_ray2 + src_spread2(lambda, L.coh_len_um));
            msum += L.E * vmf(d, f3(L.dir[0], L.dir[1], L.dir[2]), kap);
          }
        }
        add_col(msum);
        done = true;
      } else {
        const float t = hh.x;
        const float eta = xfv.w;  // |k| = eta k0 in the current medium
        footprint_update(t, kw * eta, beta2, rho);
        if (ANISO) {
          const float zb = t * 1e6f / (kw * eta);
          K.i11 += zb;
          K.i22 += zb;
        }
        const float3 x = o + t * d;
        const int mat = S.tri_mat[hslot];
        const gr_material M = S.mats[mat];
        if (M.type == GR_MAT_EMITTER && HERO) {
          // the hit measured at every class wavelength with its footprint; with
          // NEE after a diffuse vertex, power heuristic over the (wavelength,
          // technique) pairs: cf_j qpre_j p_{j,lobe} = cf_j q_j pb, cf_j qpre_j
          // p_{j,emitter}; else balance over the wavelengths
          const int ei = S.emitter_of_mat[mat];
          const float4 u = rng4(p.seed, V.view_index, pixel, smp, seg, kCallEmitFoot);
          const bool two = (p.flags & GR_FLAG_NEE) && !prev_delta && S.n_emitters > 0;
          float cf[4], qp[4] = {1.0f, 1.0f, 1.0f, 1.0f}, pb = 0.0f, den = 0.0f;
          class_shares(V, cls, Qv, cf);
          const float3 ne = emitter_normal(S, ei);
          if (two) {
            const float4 mi = P.mis[slot];  // (r2, g, kl2, cos) of the rough vertex that sampled d
            pb = rough_density(mi.y, mi.z, mi.x) * mi.w;
            const float4 q4 = P.hqp[slot];
            qp[0] = q4.x, qp[1] = q4.y, qp[2] = q4.z, qp[3] = q4.w;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if (two) {
              const float lj = step_lambda(V, cstep, cls + j * Qv), kj = 2.0f * kPi * __frcp_rn(lj);
              const float kap = 1.0f / (1.0f / (2.0f * V.beta0 * V.beta0 * kj * kj) + src_spread2(lj, M.coh_len_um));
              const float a = cf[j] * hq[j] * pb, b = cf[j] * qp[j] * vmf(-d, ne, kap) / (float)S.n_emitters;
              den += a * a + b * b;
            } else {
              den += cf[j] * hq[j];
            }
          }
#pragma unroll
          for (int g = 0; g < 4; ++g) {
            if (!(cf[g] * hq[g] > 0.0f) || !(den > 0.0f)) continue;
            const float lg = step_lambda(V, cstep, cls + g * Qv);
            float fbg = beta2, frg = rho;  // the member's footprint at the hit
            if (g != gh) member_footprint(rho, lg * __frcp_rn(lambda), V.beta0 * V.beta0, fbg, frg);
            const float mg = hero_measure_emitter(S, ei, x, d, fbg, frg, 2.0f * kPi * __frcp_rn(lg), lg, u.x, u.y);
            const float w = two ? cf[g] * cf[gh] * hq[g] * pb * pb / den : cf[g] * hq[g] / den;
            add_member(g, mg * w);
          }
          done = true;
        } else if (M.type == GR_MAT_EMITTER) {
          const int ei = S.emitter_of_mat[mat];
          float4 u = rng4(p.seed, V.view_index, pixel, smp, seg, kCallEmitFoot);
          float val = ANISO ? measure_emitter_aniso(S, ei, x, d, K, xyz(xfv), kw, lambda, u.x, u.y)
                            : measure_emitter(S, ei, x, d, beta2, rho, kw, lambda, u.x, u.y);
          float w = 1.0f;
          if ((p.flags & GR_FLAG_NEE) && !prev_delta && S.n_emitters > 0 && val > 0.0f) {
            const float3 ne = emitter_normal(S, ei);
            const float kap = 1.0f / (s_ray2 + src_spread2(lambda, M.coh_len_um));
            const float pn = vmf(-d, ne, kap) / (float)S.n_emitters;
            const float4 mi = P.mis[slot];  // (r2, g, kl2, cos) of the rough vertex that sampled d
            const float pb = rough_density(mi.y, mi.z, mi.x) * mi.w;
            w = pb * pb / (pb * pb + pn * pn);
          }
          add_col(val * w);
          done = true;
        } else if (M.type == GR_MAT_ABSORBER || seg >= V.max_depth) {
          done = true;
        } else {
          if ((p.flags & GR_FLAG_RR) && seg >= 3) {
            const float q = fminf(1.0f, fmaxf(0.05f, T[0][0]));
            float4 u = rng4(p.seed, V.view_index, pixel, smp, seg, kCallRR);
            if (u.x >= q) {
              done = true;
            } else {
              const float iq = 1.0f / q;
              for (int r = 0; r < (NS == 1 ? 1 : 4); ++r)
                for (int c = 0; c < (NS == 1 ? 1 : 4); ++c) T[r][c] *= iq;
            }
          }
          if (!done) {
            // --- interaction with the reversed wavevector
            if (HERO) {
              // the density ratios before this vertex's decision and the
              // footprints at the vertex, for its next-event estimate and for
              // an emitter hit by the direction it samples
              // (the ratios are read only at a rough vertex's next-event
              // estimate and at an emitter hit after a diffuse rough lobe)
              if (M.type == GR_MAT_ROUGH) P.hqp[slot] = make_float4(hq[0], hq[1], hq[2], hq[3]);
            }
            const float4 v0 = __ldg(&S.tri[3 * hslot]), v1 = __ldg(&S.tri[3 * hslot + 1]),
                         v2 = __ldg(&S.tri[3 * hslot + 2]);
            float3 nrm = normalize(cross(xyz(v1) - xyz(v0), xyz(v2) - xyz(v0)));
            // the front (counter-clockwise) face looks outward (into air for a dielectric)
            const bool entering = !(dot(nrm, d) > 0.0f);
            if (!entering) nrm = -nrm;
            const float cos_i = -dot(d, nrm);
            const float4 u = rng4(p.seed, V.view_index, pixel, smp, seg, kCallLobe);
            FresnelM F{1.0f, 0.0f, 1.0f, 0.0f};
            bool refracted = false;
            float cos_t = 0.0f, n_rel = 1.0f, eta_next = eta;
            if (M.type == GR_MAT_DIELECTRIC) {
              const float eta_m = M.n_re + M.cauchy_b_um2 / (lambda * lambda);
              n_rel = entering ? eta_m : 1.0f / eta_m;
              F = dielectric_pick(cos_i, n_rel, u.x, refracted, cos_t);
              if (refracted) eta_next = entering ? eta_m : 1.0f;
            } else if (M.fresnel == 1) {
              F = fresnel_conductor(cos_i, M.n_re, M.n_im);
            }
            float cn[4];
            float3 s_o = f3(0.f, 0.f, 0.f);
            if (NS == 1) {
              T[0][0] *= F.a;
              cn[0] = T[0][0];
              if (ANISO) s_o = s_vector(nrm, -d, xyz(xfv));
            } else {
              const float3 k_o = -d;
              const float3 xf = xyz(xfv);
              s_o = s_vector(nrm, k_o, xf);
              const float3 p_o = cross(k_o, s_o);
              const float cphi = dot(xf, s_o), sphi = dot(xf, p_o);
              const float r2 = cphi * cphi + sphi * sphi;
              const float c2 = (cphi * cphi - sphi * sphi) / r2, s2 = 2.0f * cphi * sphi / r2;
              for (int r = 0; r < 4; ++r) {
                const float X0 = T[r][0], X3 = T[r][3];
                const float X1 = T[r][1] * c2 - T[r][2] * s2;
                const float X2 = T[r][1] * s2 + T[r][2] * c2;
                T[r][0] = F.a * X0 + F.b * X1;
                T[r][1] = F.b * X0 + F.a * X1;
                T[r][2] = F.cr * X2 - F.ci * X3;
                T[r][3] = F.ci * X2 + F.cr * X3;
                cn[r] = T[r][0];
              }
            }
            // --- sample the scattered distribution
            const float3 t_mir = d - dot(d, nrm) * nrm;
            float3 d_out = d;
            int delta = 1;
            float4 mis_rec = make_float4(0.0f, 0.0f, 1.0f, 0.0f);
            bool alive = true;
            float g_r = 0.0f;
            if (M.type == GR_MAT_GRATING) {
              float3 gt = f3(M.gdir[0], M.gdir[1], M.gdir[2]);
              gt = gt - dot(gt, nrm) * nrm;
              if (dot(gt, gt) < 1e-12f) {
                float3 e1, e2;
                onb(nrm, e1, e2);
                gt = e1;
              }
              gt = normalize(gt);
              const float step = lambda / M.period_um;
              const TableRow row = rows[V.table_base + mat * V.nb + bin];
              const int jm = row.jmax;
              const bool renorm = !(p.flags & GR_FLAG_NO_RENORM);
              // the table's pick; within its rounding of a CDF boundary the
              // FP32 copy decides, and within FP32's rounding FP64 does
              bool ambiguous;
              int pick = grating_pick_tab(jm, t_mir, step, gt, renorm, u.x, TableRound<TT>::rel, TableRound<TT>::abs,
                                          [&](int a) { return table_load<TT>(tvals, row.offset + a); }, ambiguous);
              if (ambiguous && sizeof(TT) != sizeof(float))
                pick = grating_pick_tab(jm, t_mir, step, gt, renorm, u.x, TableRound<float>::rel,
                                        TableRound<float>::abs,
                                        [&](int a) { return __ldg(p.table_vals32 + row.offset + a); }, ambiguous);
              if (ambiguous) {
                atomicAdd(&p.ctr->ref_lobe, 1ull);
                pick = grating_pick_fp64(bin_lambda_d(V, bin), M.height_um, jm, t_mir, step, gt, renorm, u.x);
              }
              if (pick == 0x7fffffff) {
                alive = false;
              } else {
                const float3 tj = t_mir + ((float)pick * step) * gt;
                d_out = tj + sqrtf(fmaxf(0.0f, 1.0f - dot(tj, tj))) * nrm;
                if (HERO) {
                  if (pick != 0) {
                    drop_companions();  // the order's direction depends on the wavelength
                  } else {
                    // order 0 leaves in the same direction at every wavelength
                    const float ph = order0_prob(row, t_mir, step, gt, renorm, p.table_vals32);
#pragma unroll
                    for (int g = 0; g < 4; ++g) {
                      if (g == gh || hq[g] == 0.0f) continue;
                      const int bg = cls + g * Qv;
                      const float p0 = order0_prob(rows[V.table_base + mat * V.nb + bg], t_mir,
                                                   bin_lambda(V, bg) / M.period_um, gt, renorm, p.table_vals32);
                      hq[g] = ph > 0.0f ? hq[g] * (p0 / ph) : 0.0f;
                    }
                  }
                }
              }
            } else if (M.type == GR_MAT_MIRROR) {
              d_out = d + (2.0f * cos_i) * nrm;
            } else if (M.type == GR_MAT_DIELECTRIC) {
              // chosen with u.x above; refraction by Snell's law in vector form
              const float e = 1.0f / n_rel;
              d_out = refracted ? e * d + (e * cos_i - cos_t) * nrm : d + (2.0f * cos_i) * nrm;
            } else {  // rough
              g_r = 2.0f * kw * M.sigma_h_um * cos_i;
              g_r *= g_r;
              float mreal;
              if (g_r > kGCont) {
                mreal = g_r;
              } else {
                float pm = expf(-g_r), cdf = pm;
                int mi = 0;
                while (u.x >= cdf && mi < 1000) {
                  ++mi;
                  pm *= g_r / (float)mi;
                  cdf += pm;
                }
                const float eps = 4e-6f + 2e-7f * (float)mi;
                if (fabsf(u.x - cdf) < eps || (mi > 0 && fabsf(u.x - (cdf - pm)) < eps) || mi >= 1000) {
                  atomicAdd(&p.ctr->ref_lobe, 1ull);
                  mi = poisson_pick_fp64(bin_lambda_d(V, bin), M.sigma_h_um, cos_i, u.x);
                }
                mreal = (float)mi;
              }
              if (mreal == 0.0f) {
                d_out = d + (2.0f * cos_i) * nrm;
              } else {
                delta = 0;
                const float kl = kw * M.corr_len_um;
                const float sig = sqrtf(2.0f * mreal) / kl;
                float z0, z1;
                box_muller(u.y, u.z, z0, z1);
                float3 e1, e2;
                onb(nrm, e1, e2);
                const float3 dt = (sig * z0) * e1 + (sig * z1) * e2;
                const float3 to = t_mir + dt;
                const float tt = dot(to, to);
                if (tt >= 1.0f) {
                  alive = false;
                } else {
                  const float cz = sqrtf(1.0f - tt);
                  d_out = to + cz * nrm;
                  mis_rec = make_float4(dot(dt, dt), g_r, kl * kl, cz);
                }
              }
              if (HERO && alive) {
                // the class wavelengths' densities of the lobe term just
                // sampled (the cosine factor is common to all of them; g
                // scales with k^2 across the class): the specular term's
                // probability e^-g here; the m >= 1 density at the sampled
                // offset by k_density, on a compacted queue of such vertices
                // (here only a fraction of a warp's lanes would run the
                // series), from the lobe terms stored for MIS, the ratios and
                // the sample
                if (mreal == 0.0f) {
#pragma unroll
                  for (int g = 0; g < 4; ++g) {
                    if (g == gh || hq[g] == 0.0f) continue;
                    const float r = lambda * __frcp_rn(step_lambda(V, cstep, cls + g * Qv));
                    const float gqg = g_r * (r * r);  // g at class wavelength g
                    hq[g] *= gqg > kGCont ? 0.0f : expf(g_r - gqg);
                  }
                } else {
                  // (only a living companion's ratio needs the series)
#pragma unroll
                  for (int g = 0; g < 4; ++g)
                    if (g != gh && hq[g] != 0.0f) want_density = true;
                }
              }
            }
            if (HERO && M.type == GR_MAT_DIELECTRIC && M.cauchy_b_um2 != 0.0f) drop_companions();
            // --- next-event estimation toward an emitter (rough lobes only)
            if (M.type == GR_MAT_ROUGH && (p.flags & GR_FLAG_NEE) && S.n_emitters > 0) {
              const float4 un = rng4(p.seed, V.view_index, pixel, smp, seg, kCallNeeDir);
              const int ne_cnt = S.n_emitters;
              int ei = (int)(un.x * (float)ne_cnt);
              if (ei > ne_cnt - 1) ei = ne_cnt - 1;
              const float3 nE = emitter_normal(S, ei);
              const gr_material EM = S.mats[S.emitters[ei].mat];
              const float kap = 1.0f / (s_ray2 + src_spread2(lambda, EM.coh_len_um));
              const float3 w = vmf_sample(-nE, kap, un.y, un.z);
              const float cos_o = dot(w, nrm);
              if (cos_o > 0.0f && g_r > 0.0f && emitter_reachable(S, ei, x, w)) {
                // the lobe density, the MIS weight and the measurement are
                // evaluated by k_shadow once the shadow ray reaches the emitter
                const float3 dtn = (w - dot(w, nrm) * nrm) - t_mir;
                const float kl = kw * M.corr_len_um;
                P.shd[slot] = make_float4(w.x, w.y, w.z, __int_as_float(ei | (seg << 16)));
                P.shc[slot] = make_float4(cn[0], NS == 4 ? cn[1] : 0.0f, NS == 4 ? cn[2] : 0.0f, NS == 4 ? cn[3] : 0.0f);
                P.shm[slot] = make_float4(dot(dtn, dtn), g_r, kl * kl, cos_o);
                if (ANISO) {
                  // the vertex's footprint in the frame of the emitter direction
                  const float3 xw = s_vector(nrm, -w, s_o);
                  const AK Kw = ak_interaction(K, xyz(xfv), d, xw, w, nrm);
                  P.nk0[slot] = make_float4(Kw.r11, Kw.r12, Kw.r22, Kw.i11);
                  P.nk1[slot] = make_float4(Kw.i12, Kw.i22, 0.0f, 0.0f);
                  P.nkf[slot] = make_float4(xw.x, xw.y, xw.z, 0.0f);
                }
                want_shadow = true;
              }
            }
            // the vertex becomes the ray origin; (beta, rho) are unchanged by
            // the interaction (Eq. K_reflection_refraction, Eq. K_grating)
            P.od0[slot] = make_float4(x.x, x.y, x.z, beta2);
            if (alive) {
              P.od1[slot] = make_float4(d_out.x, d_out.y, d_out.z, rho);
              if (NS == 1) {
                P.tp[0][slot] = make_float4(T[0][0], eta_next, 0.0f, 0.0f);
              } else {
                for (int r = 0; r < 4; ++r) P.tp[r][slot] = make_float4(T[r][0], T[r][1], T[r][2], T[r][3]);
                const float3 xn = s_vector(nrm, -d_out, s_o);
                P.xf[slot] = make_float4(xn.x, xn.y, xn.z, eta_next);
              }
              if (!delta) P.mis[slot] = mis_rec;
              if (HERO) P.hq[slot] = make_float4(hq[0], hq[1], hq[2], hq[3]);
              if (ANISO) {
                // the footprint mapped onto the outgoing direction's frame
                const float3 xn = s_vector(nrm, -d_out, s_o);
                const AK Ko = ak_interaction(K, xyz(xfv), d, xn, d_out, nrm);
                P.ak0[slot] = make_float4(Ko.r11, Ko.r12, Ko.r22, Ko.i11);
                P.ak1[slot] = make_float4(Ko.i12, Ko.i22, 0.0f, 0.0f);
                if (NS == 1) P.xf[slot] = make_float4(xn.x, xn.y, xn.z, 0.0f);
              }
              P.meta[slot] = make_int4(m.x, m.y, meta_pack(kk, seg + 1, ST_ACTIVE, delta), hslot);
            } else {
              P.od1[slot] = make_float4(d.x, d.y, d.z, rho);
              P.meta[slot] = make_int4(m.x, m.y, meta_pack(kk, seg, ST_DONE, 0), hslot);
              // a pending next-event ray is measured in the next iteration:
              // the fold waits for it
              P.st8[slot] = want_shadow ? ST_WAIT : ST_DONE;
            }
          }
        }
      }
      P.part[slot] = pt;
      if (done) {
        P.meta[slot] = make_int4(m.x, m.y, meta_pack(kk, seg, ST_DONE, 0), m.w);
        P.st8[slot] = ST_DONE;
      }
    }
    if (HERO) {
      // the next-event and density queues with one set of barriers
      const int2 q = block_reserve2(&p.ctr->sq_count, want_shadow, &p.ctr->dq_count, want_density);
      if (want_shadow) P.sq[q.x] = slot;
      if (want_density) P.dq[q.y] = slot;
    } else {
      const int q = block_reserve<int>(&p.ctr->sq_count, want_shadow);
      if (want_shadow) P.sq[q] = slot;
    }
  }
}

// Hero-wavelength MIS: completes the density ratios q_j of the rough
// vertices k_shade queued, with the lobe's m >= 1 density at the four class
// wavelengths (rough_density_class) -- the same arithmetic on the same inputs
// as inline, on a dense queue.  Runs after k_shade, before the next
// iteration's k_shadow measures the vertices' next-event rays.
__global__ void __launch_bounds__(256) k_density(RenderParams p) {
  const Pool& P = p.pool;
  const int n = *(volatile int*)&p.ctr->dq_count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = P.dq[i];
    // the vertex's lobe terms (squared offset, g, (k l)^2 at the hero's
    // wavelength), its ratios, and the sample's class and hero member
    const float4 mi = P.mis[slot];
    const float4 q4 = P.hq[slot];
    float hq[4] = {q4.x, q4.y, q4.z, q4.w};
    const int4 m = P.meta[slot];
    const DevView& V = p.views[m.x];
    const int cls = m.y / (V.W * V.H);
    const int Qv = V.Q;
    const int bin = (class_first_sample(V, cls, Qv) + meta_k(m.z) * Qv) % V.nb;
    const int gh = (bin - cls) / Qv;
    const float lambda = bin_lambda(V, bin), cstep = bin_step(V);
    // g and (k l)^2 scale with k^2 across the class (as k_shade forms them)
    float gq[4], klq[4];
    bool want[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float r = j == gh ? 1.0f : lambda * __frcp_rn(step_lambda(V, cstep, cls + j * Qv));
      const float sc = r * r;
      gq[j] = mi.y * sc;
      klq[j] = mi.z * sc;
      want[j] = j == gh || hq[j] != 0.0f;
    }
    float dens[4];
    rough_density_class(gq, klq, want, mi.x, dens);
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      if (g == gh || hq[g] == 0.0f) continue;
      hq[g] = dens[gh] > 0.0f ? hq[g] * (dens[g] / dens[gh]) : 0.0f;
    }
    P.hq[slot] = make_float4(hq[0], hq[1], hq[2], hq[3]);
  }
}

// ------------------------------------------------------------------ shadow
// Next-event contribution of a finished shadow ray: if it reached the emitter
// it was aimed at, the emitter is measured after the segment's footprint
// update and the rough lobe's value is weighted against the emitter sampler
// by the power heuristic (the NEE request and lobe terms were stored by
// k_shade), and the result is added to the slot's sample contribution.
template <int NS, bool ANISO>
__device__ __forceinline__ void shadow_finish(const RenderParams& p, int slot, const Hit& h) {
  const Pool& P = p.pool;
  const int4 m = P.meta[slot];
  const DevView& V = p.views[m.x];
  const DevScene& S = p.scenes[V.scene_index];
  const float4 sd = P.shd[slot];
  const int tag = __float_as_int(sd.w);
  const int ei = tag & 0xffff, seg = tag >> 16;
  if (h.slot < 0 || S.tri_mat[h.slot] != S.emitters[ei].mat) return;
  const float4 a0 = P.od0[slot], a1 = P.od1[slot];
  const float3 x = xyz(a0), w = xyz(sd);
  const int WH = V.W * V.H;
  const int cls = m.y / WH;
  const int pixel = m.y - cls * WH;
  const int smp = class_first_sample(V, cls, V.Q) + meta_k(m.z) * V.Q;
  const int bin = V.Q == V.nb ? cls : smp % V.nb;  // the hero's bin under hero-wavelength MIS
  const float lambda = bin_lambda(V, bin);
  const float kw = 2.0f * kPi / lambda;
  float b2 = a0.w, ro = a1.w;
  // |k| = eta k0 in the ray's medium: air on the camera segment, else the
  // index carried with the path's throughput (scalar) or Stokes frame
  const float eta = seg == 0 ? 1.0f : (NS == 1 ? P.tp[0][slot].y : P.xf[slot].w);
  const float4 u = rng4(p.seed, V.view_index, pixel, smp, seg, kCallNeeFoot);
  float val;
  if (ANISO) {
    // the footprint stored by k_shade in the frame of w, propagated
    const float4 k0 = P.nk0[slot], k1 = P.nk1[slot], xw = P.nkf[slot];
    AK Kw{k0.x, k0.y, k0.z, k0.w, k1.x, k1.y};
    const float zb = h.t * 1e6f / (kw * eta);
    Kw.i11 += zb;
    Kw.i22 += zb;
    val = measure_emitter_aniso(S, ei, x + h.t * w, w, Kw, xyz(xw), kw, lambda, u.x, u.y);
  } else {
    footprint_update(h.t, kw * eta, b2, ro);
    val = measure_emitter(S, ei, x + h.t * w, w, b2, ro, kw, lambda, u.x, u.y);
  }
  if (val == 0.0f) return;
  // lobe density toward w and the power-heuristic weight against the
  // emitter's direction sampler
  const float4 sm = P.shm[slot];
  const float f = rough_density(sm.y, sm.z, sm.x) * sm.w;
  const float3 nE = emitter_normal(S, ei);
  const float s_ray2 = 1.0f / (2.0f * V.beta0 * V.beta0 * kw * kw);
  const float kap = 1.0f / (s_ray2 + src_spread2(lambda, S.mats[S.emitters[ei].mat].coh_len_um));
  const float pn = vmf(w, -nE, kap) / (float)S.n_emitters;
  if (f > 0.0f && pn > 0.0f) {
    const float wm = pn * pn / (pn * pn + f * f) * (f / pn) * val;
    const float4 c = P.shc[slot];
    float4 pt = P.part[slot];
    pt.x += c.x * wm;
    if (NS == 4) {
      pt.y += c.y * wm;
      pt.z += c.z * wm;
      pt.w += c.w * wm;
    }
    P.part[slot] = pt;
  }
}

// The same with hero-wavelength MIS: the estimate is measured at every class
// wavelength (footprints of the vertex, stored by k_shade) and weighted by
// the power heuristic over the (wavelength j, technique) pairs, with full
// path densities cf_j qpre_j p_{j,lobe}(w) and cf_j qpre_j p_{j,emitter}(w);
// a class wavelength's lobe density scales the hero's g and (k l)^2 by
// (k_j / k)^2.
template <int NS>
__device__ __forceinline__ void shadow_finish_hero(const RenderParams& p, int slot, const Hit& h) {
  const Pool& P = p.pool;
  const int4 m = P.meta[slot];
  const DevView& V = p.views[m.x];
  const DevScene& S = p.scenes[V.scene_index];
  const float4 sd = P.shd[slot];
  const int tag = __float_as_int(sd.w);
  const int ei = tag & 0xffff, seg = tag >> 16;
  if (h.slot < 0 || S.tri_mat[h.slot] != S.emitters[ei].mat) return;
  const float3 x = xyz(P.od0[slot]), w = xyz(sd);
  const int WH = V.W * V.H;
  const int cls = m.y / WH;
  const int pixel = m.y - cls * WH;
  const int Qv = V.Q;
  const int smp = class_first_sample(V, cls, Qv) + meta_k(m.z) * Qv;
  const int bin = smp % V.nb;
  const int gh = (bin - cls) / Qv;
  const float lambda = bin_lambda(V, bin);
  const float cstep = bin_step(V);
  const float eta = seg == 0 ? 1.0f : (NS == 1 ? P.tp[0][slot].y : P.xf[slot].w);
  const float3 nE = emitter_normal(S, ei);
  const float lc = S.mats[S.emitters[ei].mat].coh_len_um;
  const float inv_ne = 1.0f / (float)S.n_emitters;
  const float4 sm = P.shm[slot];  // squared offset, g, (k l)^2, cos of the hero's lobe toward w
  const float4 q4 = P.hqp[slot];
  const float qp[4] = {q4.x, q4.y, q4.z, q4.w};
  float cf[4], pbw[4], gq[4], klq[4], pn_h = 0.0f, den = 0.0f;
  bool want[4];
  class_shares(V, cls, Qv, cf);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float r = j == gh ? 1.0f : lambda * __frcp_rn(step_lambda(V, cstep, cls + j * Qv));
    const float sc = r * r;  // (k_j / k)^2
    gq[j] = sm.y * sc;
    klq[j] = sm.z * sc;
    want[j] = cf[j] * qp[j] > 0.0f;
  }
  rough_density_class(gq, klq, want, sm.x, pbw);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    pbw[j] *= sm.w;
    const float cq = cf[j] * qp[j];
    if (!(cq > 0.0f)) continue;
    const float lj = step_lambda(V, cstep, cls + j * Qv), kj = 2.0f * kPi * __frcp_rn(lj);
    const float kap = 1.0f / (1.0f / (2.0f * V.beta0 * V.beta0 * kj * kj) + src_spread2(lj, lc));
    const float pn = vmf(w, -nE, kap) * inv_ne;
    if (j == gh) pn_h = pn;
    den += cq * cq * (pbw[j] * pbw[j] + pn * pn);
  }
  if (!(pn_h > 0.0f) || !(den > 0.0f)) return;
  // the vertex's footprint: the hero's (rho stored with the ray; beta^2 with
  // its origin) and the members' from it (member_footprint)
  const float rho_v = P.od1[slot].w, b2_v = P.od0[slot].w;
  const float4 u = rng4(p.seed, V.view_index, pixel, smp, seg, kCallNeeFoot);
  const float4 c = P.shc[slot];
#pragma unroll
  for (int g = 0; g < 4; ++g) {
    if (!(pbw[g] > 0.0f)) continue;
    const float lg = step_lambda(V, cstep, cls + g * Qv), kg = 2.0f * kPi * __frcp_rn(lg);
    float b2 = b2_v, ro = rho_v;
    if (g != gh) member_footprint(rho_v, lg * __frcp_rn(lambda), V.beta0 * V.beta0, b2, ro);
    footprint_update_ik(h.t, lg * kInv2Pi * __frcp_rn(eta), b2, ro);
    const float mg = hero_measure_emitter(S, ei, x + h.t * w, w, b2, ro, kg, lg, u.x, u.y);
    const float val = mg * cf[g] * cf[gh] * qp[g] * pn_h * pbw[g] / den;
    if (val == 0.0f) continue;
    if (g != gh) {
      member_add<NS>(P, (size_t)p.P, g, slot, c.x, c.y, c.z, c.w, val);
      continue;
    }
    float4 pt = P.part[slot];
    pt.x += c.x * val;
    if (NS == 4) {
      pt.y += c.y * val;
      pt.z += c.z * val;
      pt.w += c.w * val;
    }
    P.part[slot] = pt;
  }
}

// Next-event measurement of the shadow rays the previous k_shade requested,
// whose closest hits this iteration's k_trace launch found: each ray that
// reached its emitter adds its MIS-weighted measurement to its slot's sample,
// before k_shade adds the sample's next segment (path order).  The last block
// to finish closes the iteration's queues: it records the trace queue for
// k_shade, the live count (traced rays and held samples) for the next regen
// pass and the loop's exit test, and empties the trace and shadow queues.
template <int NS, int MODE>
__global__ void __launch_bounds__(256) k_shadow(RenderParams p) {
  const Pool& P = p.pool;
  __shared__ int s_n;
  if (threadIdx.x == 0) s_n = *(volatile int*)&p.ctr->sq_count;
  __syncthreads();
  const int n = s_n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int slot = P.sq[i];
    const float2 hh = P.shh[slot];
    Hit h;
    h.t = hh.x;
    h.slot = __float_as_int(hh.y);
    if (MODE == 1)
      shadow_finish_hero<NS>(p, slot, h);
    else
      shadow_finish<NS, MODE == 2>(p, slot, h);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // every block has read sq_count before it counts itself here
    __threadfence();
    if (atomicAdd(&p.ctr->sq_done, 1) == (int)gridDim.x - 1) {
      __threadfence();
      Counters* c = p.ctr;
      const int front = *(volatile int*)&c->tq_count;
      const int nt = front + *(volatile int*)&c->tq_back;
      c->shadow += (unsigned long long)n;
      c->tq_front = front;
      c->tq_n = nt;
      c->last_active = nt + (int)c->held;
      c->tq_count = 0;
      c->tq_back = 0;
      c->trace_next = 0;
      c->held = 0;
      c->sq_count = 0;
      c->sq_done = 0;
    }
  }
}

// ------------------------------------------------------------------ order tables
struct TableBuildRow {
  int offset, jmax, view, bin;
  float height_um;
  int pad[3];
};

// Order weight a_j = J_j(x)^2 at x = pi h / lambda (Eq. K_grating), the
// Bessel function in FP64, rounded once to FP32; tables of narrower types
// round that value to nearest.
__device__ __forceinline__ float order_weight(int j, double x) {
  const double J = bessel_j_d(j, x);
  return (float)(J * J);
}
template <typename TT>
__device__ __forceinline__ TT table_store(float v);
template <>
__device__ __forceinline__ float table_store<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half table_store<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 table_store<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// vals32 (FP32 copy for re-decisions) is null when TT is float.
template <typename TT>
__global__ void k_tables(const TableBuildRow* rows, int n_rows, const DevView* views, TT* vals, float* vals32) {
  int r = blockIdx.x;
  if (r >= n_rows) return;
  const TableBuildRow R = rows[r];
  const DevView& V = views[R.view];
  const double lam = bin_lambda_d(V, R.bin);
  const double x = kPiD * (double)R.height_um / lam;  // h k / 2
  for (int j = threadIdx.x; j <= R.jmax; j += blockDim.x) {
    const float v = order_weight(j, x);
    vals[R.offset + j] = table_store<TT>(v);
    if (vals32) vals32[R.offset + j] = v;
  }
}

// ------------------------------------------------------------------ readback
__global__ void k_readback(const float* __restrict__ sum, const float* __restrict__ comp, int W, int H, int nb, int ns,
                           const float* __restrict__ inv_count, float* __restrict__ out) {
  const long long n = (long long)W * H * nb * ns;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    // out layout [y][x][bin][stokes]; accumulator layout [bin][y][x][stokes]
    const int s = (int)(i % ns);
    long long r = i / ns;
    const int b = (int)(r % nb);
    const long long pix = r / nb;
    const long long a = ((long long)b * W * H + pix) * ns + s;
    out[i] = (sum[a] - comp[a]) * inv_count[b];
  }
}

// Condition of the single-launch render graph: repeat the iteration while any
// slot is live or tickets remain; stop (and flag) at the iteration bound.
__global__ void k_loop_cond(Counters* ctr, cudaGraphConditionalHandle h, long long max_iter) {
  bool more = !(ctr->last_active == 0 && ctr->next_ticket >= ctr->total_tickets);
  if (more && (long long)ctr->iters >= max_iter) {
    ctr->err = 3;
    more = false;
  }
  if (ctr->err) more = false;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}

// Camera basis of every view from its descriptor (pinhole: forward, right =
// forward x up, up' = right x forward, tan of half the vertical FOV).
__global__ void k_views(const gr_view_desc* __restrict__ vd, DevView* views, int n) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= n) return;
  const gr_view_desc d = vd[v];
  DevView& V = views[v];
  const float3 eye = f3(d.eye[0], d.eye[1], d.eye[2]);
  const float3 fw = normalize(f3(d.look_at[0], d.look_at[1], d.look_at[2]) - eye);
  const float3 rt = normalize(cross(fw, f3(d.up[0], d.up[1], d.up[2])));
  V.eye = eye;
  V.fw = fw;
  V.right = rt;
  V.upc = cross(rt, fw);
  V.th = tanf(0.5f * d.vfov_deg * kPi / 180.0f);
  V.aspect = (float)d.width / (float)d.height;
}

__global__ void k_debug_rng(uint32_t seed, uint32_t view, uint32_t pixel, uint32_t sample, int seg, int call, int n,
                            uint4* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = philox10(make_uint4(pixel, sample + (uint32_t)i, ((uint32_t)seg << 4) | (uint32_t)call, 0u), seed, view);
}

cudaError_t debug_rng_impl(uint32_t seed, uint32_t view, uint32_t pixel, uint32_t sample, int seg, int call, int n,
                           uint32_t* host_out, cudaStream_t st) {
  uint4* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(uint4) * (size_t)n, st);
  if (e != cudaSuccess) return e;
  k_debug_rng<<<(n + 255) / 256, 256, 0, st>>>(seed, view, pixel, sample, seg, call, n, d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d, sizeof(uint4) * (size_t)n, cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// Inspection: one order-table row as the render stores it, decoded to float.
template <typename TT>
__global__ void k_debug_table(double x, int jmax, float* out) {
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j <= jmax; j += gridDim.x * blockDim.x) {
    const TT v = table_store<TT>(order_weight(j, x));
    out[j] = table_load<TT>(&v, 0);
  }
}

cudaError_t debug_table_impl(float height_um, double lambda_um, int jmax, int dtype, float* host_out,
                             cudaStream_t st) {
  float* d = nullptr;
  cudaError_t e = cudaMallocAsync(&d, sizeof(float) * (size_t)(jmax + 1), st);
  if (e != cudaSuccess) return e;
  const double x = kPiD * (double)height_um / lambda_um;  // pi h / lambda, as in k_tables
  const int grid = (jmax + 256) / 256;
  if (dtype == GR_TABLE_F32)
    k_debug_table<float><<<grid, 256, 0, st>>>(x, jmax, d);
  else if (dtype == GR_TABLE_F16)
    k_debug_table<__half><<<grid, 256, 0, st>>>(x, jmax, d);
  else
    k_debug_table<__nv_bfloat16><<<grid, 256, 0, st>>>(x, jmax, d);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, d, sizeof(float) * (size_t)(jmax + 1), cudaMemcpyDeviceToHost, st);
  cudaFreeAsync(d, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// Inspection: the footprint update the path applies after each segment.
__global__ void k_debug_footprint(int n, const float4* in, float2* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float4 q = in[i];  // beta^2 (um^2), rho, t (m), kw (1/um)
    float beta2 = q.x, rho = q.y;
    footprint_update(q.z, q.w, beta2, rho);
    out[i] = make_float2(beta2, rho);
  }
}

cudaError_t debug_footprint_impl(int n, const float* host_in, float* host_out, cudaStream_t st) {
  float4* din = nullptr;
  float2* dout = nullptr;
  cudaError_t e = cudaMallocAsync(&din, sizeof(float4) * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dout, sizeof(float2) * (size_t)n, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(din, host_in, sizeof(float4) * (size_t)n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_debug_footprint<<<std::min((n + 255) / 256, 4096), 256, 0, st>>>(n, din, dout);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(host_out, dout, sizeof(float2) * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (din) cudaFreeAsync(din, st);
  if (dout) cudaFreeAsync(dout, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return e;
}

// ================================================================== host side
namespace {

int sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Block size of the binary-tree trace kernel for a render's block size.
int trace_block(int block) { return block < GR_TRACE_BLOCK ? block : GR_TRACE_BLOCK; }

// Blocks of k_shadow: its queue is the few next-event rays of one iteration
// (two blocks per SM cover the usual case in one pass), and every block takes
// part in closing the queues, so the grid stays small.
#ifndef GR_SHADOW_BLOCKS_PER_SM
#define GR_SHADOW_BLOCKS_PER_SM 2
#endif
int shadow_grid(long long P, int sms) {
  return (int)std::min<long long>((P + 255) / 256, (long long)GR_SHADOW_BLOCKS_PER_SM * sms);
}

// One wavefront iteration: regen, trace (with the previous shade's next-event
// rays), shadow (their measurement), shade.  With `ev` (profiling) an event
// is recorded before each kernel and after the last, so each kernel's device
// time is measured on the stream it runs on.

template <int NS, typename TT, int TREE>
cudaError_t launch_iteration_t(const RenderParams& p, int grid_regen, int grid_trace, int grid_shade, int grid_shadow,
                               int block, size_t smem, cudaStream_t st, cudaEvent_t* ev) {
  const bool hero = (p.flags & GR_FLAG_HERO) != 0, aniso = (p.flags & GR_FLAG_ANISO) != 0;
  if (ev) cudaEventRecord(ev[0], st);
  if (hero)
    k_regen<NS, true><<<grid_regen, block, 0, st>>>(p);
  else
    k_regen<NS, false><<<grid_regen, block, 0, st>>>(p);
  if (ev) cudaEventRecord(ev[1], st);
  k_trace<TREE><<<grid_trace, TREE == kTreeWide ? block : trace_block(block), 0, st>>>(p);
  if (ev) cudaEventRecord(ev[2], st);
  if (hero)
    k_shadow<NS, 1><<<grid_shadow, 256, 0, st>>>(p);
  else if (aniso)
    k_shadow<NS, 2><<<grid_shadow, 256, 0, st>>>(p);
  else
    k_shadow<NS, 0><<<grid_shadow, 256, 0, st>>>(p);
  if (ev) cudaEventRecord(ev[3], st);
  if (hero) {
    k_shade<NS, TT, 1><<<grid_shade, block, smem, st>>>(p);
    k_density<<<grid_shade, 256, 0, st>>>(p);  // counted with shading
  } else if (aniso)
    k_shade<NS, TT, 2><<<grid_shade, block, smem, st>>>(p);
  else
    k_shade<NS, TT, 0><<<grid_shade, block, smem, st>>>(p);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError();
}

template <int NS, typename TT>
cudaError_t launch_iteration(const RenderParams& p, int tree, int grid_regen, int grid_trace, int grid_shade,
                             int grid_shadow, int block, size_t smem, cudaStream_t st, cudaEvent_t* ev) {
  if (tree == kTreeWide)
    return launch_iteration_t<NS, TT, kTreeWide>(p, grid_regen, grid_trace, grid_shade, grid_shadow, block, smem, st, ev);
  if (tree == kTreeHalf)
    return launch_iteration_t<NS, TT, kTreeHalf>(p, grid_regen, grid_trace, grid_shade, grid_shadow, block, smem, st, ev);
  return launch_iteration_t<NS, TT, kTreeF32>(p, grid_regen, grid_trace, grid_shade, grid_shadow, block, smem, st, ev);
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// The shade, regen and shadow kernels a render launches (for occupancy
// queries); mode 0 plain, 1 hero-wavelength MIS, 2 anisotropic footprints.
template <int NS, typename TT>
const void* shade_kernel_t(int mode) {
  return mode == 1 ? (const void*)k_shade<NS, TT, 1> : mode == 2 ? (const void*)k_shade<NS, TT, 2>
                                                                 : (const void*)k_shade<NS, TT, 0>;
}
const void* shade_kernel(int ns, int dtype, int mode) {
  if (ns == 1) {
    if (dtype == GR_TABLE_F32) return shade_kernel_t<1, float>(mode);
    if (dtype == GR_TABLE_F16) return shade_kernel_t<1, __half>(mode);
    return shade_kernel_t<1, __nv_bfloat16>(mode);
  }
  if (dtype == GR_TABLE_F32) return shade_kernel_t<4, float>(mode);
  if (dtype == GR_TABLE_F16) return shade_kernel_t<4, __half>(mode);
  return shade_kernel_t<4, __nv_bfloat16>(mode);
}
const void* trace_kernel(int tree) {
  return tree == kTreeWide ? (const void*)k_trace<kTreeWide>
                           : tree == kTreeHalf ? (const void*)k_trace<kTreeHalf> : (const void*)k_trace<kTreeF32>;
}
// The tree a render walks: the 4-wide one on request, else the FP16 binary
// nodes unless FP32 nodes are requested or a scene has no FP16 nodes (its
// coordinates exceed the FP16 range; scenes of fewer than 2 triangles need no
// nodes).
int pick_tree(int flags, gr_scene* const* scenes, int n_scenes) {
  if (flags & GR_FLAG_WIDE_BVH) return kTreeWide;
  if (flags & GR_FLAG_FP32_NODES) return kTreeF32;
  for (int i = 0; i < n_scenes; ++i)
    if (scenes[i]->n_tris >= 2 && !scenes[i]->dev.hnodes) return kTreeF32;
  return kTreeHalf;
}
const void* regen_kernel(int ns, bool hero) {
  if (ns == 1) return hero ? (const void*)k_regen<1, true> : (const void*)k_regen<1, false>;
  return hero ? (const void*)k_regen<4, true> : (const void*)k_regen<4, false>;
}

}  // namespace

struct RenderPlan {
  std::vector<DevView> views;
  std::vector<DevScene> scenes;
  std::vector<TableRow> rows;
  std::vector<TableBuildRow> build_rows;
  int vals_count = 0;
  unsigned long long total_tickets = 0;
  long long hero_classes = 0;  // class records of views whose classes are split (hs > 1)
};

// Called by gr_render after argument validation.
// acc_sum[v] / acc_comp[v]: view v's accumulator planes; f supplies the
// scratch, counters and graph cache of the call.
// With plan_bytes != nullptr nothing is enqueued: the scratch size the render
// would hold is written there (f may then be null; acc_sum/acc_comp unused).
gr_status render_impl(gr_scene* const* scenes, int n_scenes, const gr_view_desc* vd_in, int n_views,
                      const gr_render_opts& o, gr_frame* f, const std::vector<float*>& acc_sum,
                      const std::vector<float*>& acc_comp, cudaStream_t st, std::string& err,
                      size_t* plan_bytes) {
  // Tickets are numbered over the views in order of decreasing path depth, so
  // that the paths still running once every ticket is claimed (the render's
  // tail) belong to the shallowest views.  Results do not depend on the
  // order: each view keeps its RNG key and its accumulators.
  std::vector<int> order(n_views);
  for (int v = 0; v < n_views; ++v) order[v] = v;
  std::stable_sort(order.begin(), order.end(),
                   [&](int a, int b) { return vd_in[a].max_depth > vd_in[b].max_depth; });
  std::vector<gr_view_desc> vds(n_views);
  for (int v = 0; v < n_views; ++v) vds[v] = vd_in[order[v]];
  const gr_view_desc* vd = vds.data();
  const int NSv = vd[0].n_stokes;
  RenderPlan plan;
  plan.scenes.resize(n_scenes);
  for (int i = 0; i < n_scenes; ++i) plan.scenes[i] = scenes[i]->dev;
  const size_t tsize = o.table_dtype == GR_TABLE_F32 ? 4 : 2;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = vd[v];
    DevView V;
    std::memset(&V, 0, sizeof V);
    // camera basis (eye, fw, right, upc, th, aspect) is filled by k_views
    V.W = d.width;
    V.H = d.height;
    V.nb = d.n_bins;
    V.ns = d.n_stokes;
    V.max_depth = d.max_depth;
    V.spp = d.spp;
    V.first_sample = d.first_sample;
    V.view_index = d.view_index;
    V.scene_index = d.scene_index;
    V.ortho = d.ortho;
    V.ortho_half = d.ortho_half_m;
    V.lmin = d.lambda_min_um;
    V.lmax = d.lambda_max_um;
    V.beta0 = d.f_beta * d.p_pix_um;
    V.ticket_base = (long long)plan.total_tickets;
    V.Q = (o.flags & GR_FLAG_HERO) ? d.n_bins / 4 : d.n_bins;
    V.nbu = std::min(d.spp, V.Q);
    // hero-wavelength MIS: a class with n samples is split into hs = min(4,
    // n) tickets of consecutive sample ranges (every class has at least
    // floor(spp / Q) samples), so the pool holds as many paths in flight as
    // the plain form's one-bin tickets; the ranges' sums meet in a class
    // record (fold_class).  hs depends on the view alone, so images do not
    // depend on the pool or on the other views.
    V.hs = 1;
    V.hbase = 0;
    if ((o.flags & GR_FLAG_HERO) && d.spp / V.Q >= 2) {
      V.hs = std::min(4, d.spp / V.Q);
      V.hbase = plan.hero_classes;
      plan.hero_classes += (long long)V.Q * d.width * d.height;
    }
    V.n_tickets = (long long)V.nbu * d.width * d.height * V.hs;
    plan.total_tickets += (unsigned long long)V.n_tickets;
    V.acc_sum = plan_bytes ? nullptr : acc_sum[order[v]];
    V.acc_comp = plan_bytes ? nullptr : acc_comp[order[v]];
    // grating order table rows for every (material, bin) of this view
    const gr_scene* sc = scenes[d.scene_index];
    V.table_base = (int)plan.rows.size();
    for (size_t m = 0; m < sc->mats.size(); ++m) {
      for (int b = 0; b < d.n_bins; ++b) {
        TableRow r{0, -1};
        const gr_material& M = sc->mats[m];
        if (M.type == GR_MAT_GRATING) {
          double lam = d.n_bins <= 1 ? (double)d.lambda_min_um
                                     : (double)d.lambda_min_um + (double)b * ((double)d.lambda_max_um - (double)d.lambda_min_um) /
                                                                     (double)(d.n_bins - 1);
          int jm = (int)std::floor(2.0 * (double)M.period_um / lam) + 2;
          if (jm > kMaxOrder) jm = kMaxOrder;
          r.offset = plan.vals_count;
          r.jmax = jm;
          plan.vals_count += jm + 1;
          TableBuildRow br{};
          br.offset = r.offset;
          br.jmax = jm;
          br.view = v;
          br.bin = b;
          br.height_um = M.height_um;
          plan.build_rows.push_back(br);
        }
        plan.rows.push_back(r);
      }
    }
    plan.views.push_back(V);
  }
  // ---- scratch layout
  const bool hero = (o.flags & GR_FLAG_HERO) != 0, aniso = (o.flags & GR_FLAG_ANISO) != 0;
  // Default pool: one slot per ticket (every ticket runs from the first
  // iteration, so the render takes the fewest iterations and launch tails),
  // capped at kMaxDefaultPool slots and at a quarter of the device memory
  // free for this frame's scratch.  Images do not depend on the pool size.
  long long P = o.pool_size;
  if (P <= 0) {
    const size_t per_slot = sizeof(float4) * 14 + 2 * sizeof(float2) + sizeof(int4) + 2 * sizeof(int) + 1 +
                            (hero ? sizeof(float4) * 10 + sizeof(int) : 0) + (aniso ? sizeof(float4) * 5 : 0);
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      free_b = 0;
    }
    const long long mem_cap = (long long)((free_b + (f ? f->scratch_bytes : 0)) / 4 / per_slot);
    P = std::min<long long>(kMaxDefaultPool, std::max<long long>(mem_cap, kMinDefaultPool));
  }
  if ((unsigned long long)P > plan.total_tickets) P = (long long)std::max<unsigned long long>(plan.total_tickets, 1ull);
  P = (P + 255) / 256 * 256;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = align_up(off + bytes, 256);
    return r;
  };
  const size_t o_views = take(sizeof(DevView) * n_views);
  const size_t o_vdesc = take(sizeof(gr_view_desc) * n_views);
  const size_t o_scenes = take(sizeof(DevScene) * n_scenes);
  const size_t o_rows = take(sizeof(TableRow) * std::max<size_t>(plan.rows.size(), 1));
  const size_t o_brows = take(sizeof(TableBuildRow) * std::max<size_t>(plan.build_rows.size(), 1));
  const size_t o_vals = take(tsize * std::max(plan.vals_count, 1));
  const size_t o_vals32 = o.table_dtype == GR_TABLE_F32 ? o_vals : take(sizeof(float) * std::max(plan.vals_count, 1));
  const size_t o_f4 = take(sizeof(float4) * (size_t)P * 14);
  const size_t o_hit = take(sizeof(float2) * (size_t)P * 2);  // hit, shh
  const size_t o_meta = take(sizeof(int4) * (size_t)P);
  const size_t o_tq = take(sizeof(int) * (size_t)P);
  const size_t o_sq = take(sizeof(int) * (size_t)P);
  const size_t o_st8 = take((size_t)P);
  const int mode = hero ? 1 : aniso ? 2 : 0;
  // hq, hqp, haccS/haccC[4], then the density queue
  const size_t o_hero = hero ? take(sizeof(float4) * (size_t)P * 10) : 0;
  const size_t o_dq = hero ? take(sizeof(int) * (size_t)P) : 0;
  // range totals of split classes: 4 ranges x 4 members x 4 Stokes floats per
  // class record, and the count of ranges folded
  const size_t o_hsub = plan.hero_classes ? take(sizeof(float) * 64 * (size_t)plan.hero_classes) : 0;
  const size_t o_hsubn = plan.hero_classes ? take(sizeof(int) * (size_t)plan.hero_classes) : 0;
  const size_t o_aniso = aniso ? take(sizeof(float4) * (size_t)P * 5) : 0;  // ak0, ak1, nk0, nk1, nkf
  const size_t total = off;
  if (plan_bytes) {
    *plan_bytes = total;
    return GR_OK;
  }
  if (f->scratch_bytes < total) {
    if (f->scratch) cudaFreeAsync(f->scratch, st);
    f->scratch = nullptr;
    f->scratch_bytes = 0;
    if (cudaMallocAsync(&f->scratch, total, st) != cudaSuccess) {
      err = "scratch allocation failed";
      return GR_E_OOM;
    }
    f->scratch_bytes = total;
  }
  unsigned char* base = (unsigned char*)f->scratch;
  RenderParams p;
  std::memset(&p, 0, sizeof p);
  p.views = (const DevView*)(base + o_views);
  p.n_views = n_views;
  p.scenes = (const DevScene*)(base + o_scenes);
  p.seed = o.seed;
  p.flags = o.flags;
  p.rows = (const TableRow*)(base + o_rows);
  p.table_vals = base + o_vals;
  p.table_vals32 = (const float*)(base + o_vals32);
  p.table_dtype = o.table_dtype;
  p.table_rows = (int)plan.rows.size();
  p.table_vals_count = plan.vals_count;
  float4* f4 = (float4*)(base + o_f4);
  p.pool.od0 = f4;
  p.pool.od1 = f4 + (size_t)P;
  for (int r = 0; r < 4; ++r) p.pool.tp[r] = f4 + (size_t)P * (2 + r);
  p.pool.xf = f4 + (size_t)P * 6;
  p.pool.part = f4 + (size_t)P * 7;
  p.pool.accS = f4 + (size_t)P * 8;
  p.pool.accC = f4 + (size_t)P * 9;
  p.pool.shd = f4 + (size_t)P * 10;
  p.pool.shc = f4 + (size_t)P * 11;
  p.pool.shm = f4 + (size_t)P * 12;
  p.pool.mis = f4 + (size_t)P * 13;
  p.pool.hit = (float2*)(base + o_hit);
  p.pool.shh = p.pool.hit + (size_t)P;
  p.pool.meta = (int4*)(base + o_meta);
  p.pool.tq = (int*)(base + o_tq);
  p.pool.sq = (int*)(base + o_sq);
  p.pool.st8 = base + o_st8;
  if (hero) {
    float4* h4 = (float4*)(base + o_hero);
    p.pool.hq = h4;
    p.pool.hqp = h4 + (size_t)P;
    p.pool.haccS = h4 + (size_t)P * 2;
    p.pool.haccC = h4 + (size_t)P * 6;
    p.pool.dq = (int*)(base + o_dq);
    if (plan.hero_classes) {
      p.pool.hsub = (float*)(base + o_hsub);
      p.pool.hsub_n = (int*)(base + o_hsubn);
    }
  }
  if (aniso) {
    float4* a4 = (float4*)(base + o_aniso);
    p.pool.ak0 = a4;
    p.pool.ak1 = a4 + (size_t)P;
    p.pool.nk0 = a4 + (size_t)P * 2;
    p.pool.nk1 = a4 + (size_t)P * 3;
    p.pool.nkf = a4 + (size_t)P * 4;
  }
  p.P = (int)P;
  p.regen_thr = o.regen_threshold_pct;
  p.ctr = f->ctr;
  const size_t smem_table = sizeof(TableRow) * plan.rows.size() + tsize * plan.vals_count;
  p.table_smem = smem_table <= 40 * 1024 ? 1 : 0;
  const size_t smem = p.table_smem ? align_up(smem_table, 16) : 0;

  cudaError_t e;
#define GR_CK(x)                                 \
  do {                                           \
    e = (x);                                     \
    if (e != cudaSuccess) {                      \
      err = std::string(#x) + ": " + cudaGetErrorString(e); \
      return GR_E_CUDA;                          \
    }                                            \
  } while (0)
  GR_CK(cudaMemcpyAsync(base + o_views, plan.views.data(), sizeof(DevView) * n_views, cudaMemcpyHostToDevice, st));
  GR_CK(cudaMemcpyAsync(base + o_vdesc, vd, sizeof(gr_view_desc) * n_views, cudaMemcpyHostToDevice, st));
  k_views<<<(n_views + 63) / 64, 64, 0, st>>>((const gr_view_desc*)(base + o_vdesc), (DevView*)(base + o_views), n_views);
  f->launches += 1;
  GR_CK(cudaMemcpyAsync(base + o_scenes, plan.scenes.data(), sizeof(DevScene) * n_scenes, cudaMemcpyHostToDevice, st));
  if (!plan.rows.empty())
    GR_CK(cudaMemcpyAsync(base + o_rows, plan.rows.data(), sizeof(TableRow) * plan.rows.size(), cudaMemcpyHostToDevice, st));
  if (!plan.build_rows.empty()) {
    GR_CK(cudaMemcpyAsync(base + o_brows, plan.build_rows.data(), sizeof(TableBuildRow) * plan.build_rows.size(),
                          cudaMemcpyHostToDevice, st));
    const TableBuildRow* br = (const TableBuildRow*)(base + o_brows);
    const int nr = (int)plan.build_rows.size();
    if (o.table_dtype == GR_TABLE_F32)
      k_tables<float><<<nr, 64, 0, st>>>(br, nr, p.views, (float*)(base + o_vals), nullptr);
    else if (o.table_dtype == GR_TABLE_F16)
      k_tables<__half><<<nr, 64, 0, st>>>(br, nr, p.views, (__half*)(base + o_vals), (float*)(base + o_vals32));
    else
      k_tables<__nv_bfloat16><<<nr, 64, 0, st>>>(br, nr, p.views, (__nv_bfloat16*)(base + o_vals), (float*)(base + o_vals32));
    f->launches += 1;
  }
  GR_CK(cudaMemsetAsync(p.pool.meta, 0, sizeof(int4) * (size_t)P, st));
  GR_CK(cudaMemsetAsync(p.pool.st8, ST_IDLE, (size_t)P, st));
  if (plan.hero_classes) GR_CK(cudaMemsetAsync(p.pool.hsub_n, 0, sizeof(int) * (size_t)plan.hero_classes, st));
  Counters c0;
  std::memset(&c0, 0, sizeof c0);
  c0.total_tickets = plan.total_tickets;
  GR_CK(cudaMemcpyAsync(f->ctr, &c0, sizeof c0, cudaMemcpyHostToDevice, st));
  GR_CK(cudaGetLastError());

  // ---- launch shapes
  const int dev = f->device;
  const int sms = sm_count(dev);
  const int block = o.block > 0 ? o.block : 256;
  auto grid_for = [&](const void* fn, size_t dyn, int blk = 0) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, blk > 0 ? blk : block, dyn);
    if (per < 1) per = 1;
    return sms * per;
  };
  int g_regen, g_trace, g_shade, g_shadow;
  const void* shade_fn = shade_kernel(NSv, o.table_dtype, mode);
  g_regen = grid_for(regen_kernel(NSv, hero), 0);
  const int tree = pick_tree(o.flags, scenes, n_scenes);
  g_shadow = shadow_grid(P, sms);
  const int tblk = tree == kTreeWide ? block : trace_block(block);
  g_trace = grid_for(trace_kernel(tree), 0, tblk);
  g_shade = grid_for(shade_fn, smem);
  // never more blocks than the pool needs
  const int gmax = (int)((P + block - 1) / block);
  g_regen = std::min(g_regen, (int)((P + (long long)block * GR_REGEN_SLOTS - 1) / ((long long)block * GR_REGEN_SLOTS)));
  g_trace = std::min(g_trace, (int)((P + tblk - 1) / tblk));
  g_shade = std::min(g_shade, gmax);

  const bool profile = o.profile && !o.use_graph;
  std::vector<cudaEvent_t> pev;
  auto launch_on = [&](cudaStream_t ls) -> cudaError_t {
    if (NSv == 1) {
      if (o.table_dtype == GR_TABLE_F32) return launch_iteration<1, float>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, ls, nullptr);
      if (o.table_dtype == GR_TABLE_F16) return launch_iteration<1, __half>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, ls, nullptr);
      return launch_iteration<1, __nv_bfloat16>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, ls, nullptr);
    }
    if (o.table_dtype == GR_TABLE_F32) return launch_iteration<4, float>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, ls, nullptr);
    if (o.table_dtype == GR_TABLE_F16) return launch_iteration<4, __half>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, ls, nullptr);
    return launch_iteration<4, __nv_bfloat16>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, ls, nullptr);
  };
  auto launch = [&]() -> cudaError_t {
    cudaEvent_t* ev = nullptr;
    if (profile) {
      size_t b = pev.size();
      for (int i = 0; i < 5; ++i) {
        cudaEvent_t e2;
        cudaEventCreate(&e2);
        pev.push_back(e2);
      }
      ev = pev.data() + b;
    }
    if (NSv == 1) {
      if (o.table_dtype == GR_TABLE_F32) return launch_iteration<1, float>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, ev);
      if (o.table_dtype == GR_TABLE_F16) return launch_iteration<1, __half>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, ev);
      return launch_iteration<1, __nv_bfloat16>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, ev);
    }
    if (o.table_dtype == GR_TABLE_F32) return launch_iteration<4, float>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, ev);
    if (o.table_dtype == GR_TABLE_F16) return launch_iteration<4, __half>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, ev);
    return launch_iteration<4, __nv_bfloat16>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, ev);
  };

  // ---- iteration loop: batches of B iterations; the host watches the
  // device's live-slot count of the batch before the last one
  const int B = 8;
  // Worst case of the schedule: each slot runs ceil(T/P) tickets one after the
  // other, each of at most n samples taking at most max_depth + 2 iterations.
  long long worst = 0;
  {
    long long n_max = 1, d_max = 0;
    for (int v = 0; v < n_views; ++v) {
      n_max = std::max<long long>(n_max, (long long)vd[v].spp / plan.views[v].Q + 1);
      d_max = std::max<long long>(d_max, vd[v].max_depth);
    }
    long long rounds = (long long)((plan.total_tickets + P - 1) / P) + 1;
    worst = rounds * n_max * (d_max + 3) + 4 * B;
  }
  const long long max_iter = o.max_iterations > 0 ? o.max_iterations : 2 * worst;
  if (o.use_graph) {
    // ---- one graph launch: conditional while-node around one iteration
    std::vector<unsigned char> key(sizeof(RenderParams) + 8 * sizeof(long long));
    long long shape[8] = {g_regen, g_trace, g_shade, g_shadow, block, (long long)smem,
                          (tree * 16 + NSv) * 16 + o.table_dtype, max_iter};
    std::memcpy(key.data(), &p, sizeof p);
    std::memcpy(key.data() + sizeof p, shape, sizeof shape);
    if (!f->graph_exec || f->graph_key != key) {
      if (f->graph_exec) cudaGraphExecDestroy(f->graph_exec);
      f->graph_exec = nullptr;
      cudaGraph_t g = nullptr;
      GR_CK(cudaGraphCreate(&g, 0));
      cudaGraphConditionalHandle h;
      e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
      cudaGraphNode_t cnode;
      cudaGraphNodeParams np = {};
      np.type = cudaGraphNodeTypeConditional;
      np.conditional.handle = h;
      np.conditional.type = cudaGraphCondTypeWhile;
      np.conditional.size = 1;
      if (e == cudaSuccess) e = cudaGraphAddNode(&cnode, g, nullptr, nullptr, 0, &np);
      // the body is recorded on a private stream (capture is not allowed on
      // the legacy default stream); the graph is then launched on `st`
      if (e == cudaSuccess && !f->capture_stream) e = cudaStreamCreateWithFlags(&f->capture_stream, cudaStreamNonBlocking);
      if (e == cudaSuccess) {
        cudaGraph_t body = np.conditional.phGraph_out[0];
        cudaStream_t cs = f->capture_stream;
        e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
          cudaError_t le = launch_on(cs);
          k_loop_cond<<<1, 1, 0, cs>>>(p.ctr, h, max_iter);
          if (le == cudaSuccess) le = cudaGetLastError();
          cudaGraph_t captured = nullptr;
          e = cudaStreamEndCapture(cs, &captured);
          if (e == cudaSuccess) e = le;
        }
      }
      if (e == cudaSuccess) e = cudaGraphInstantiate(&f->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) {
        f->graph_exec = nullptr;
        err = std::string("render graph: ") + cudaGetErrorString(e);
        return GR_E_CUDA;
      }
      f->graph_key = key;
    }
    GR_CK(cudaGraphLaunch(f->graph_exec, st));
    Counters* hc = f->ctr_host;
    GR_CK(cudaMemcpyAsync(hc, f->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st));
    GR_CK(cudaStreamSynchronize(st));
    f->iterations += (long long)hc->iters;
    f->launches += (5LL + (hero ? 1 : 0)) * (long long)hc->iters + 1;
    if (hc->err == 3) {
      err = "render exceeded its iteration bound";
      return GR_E_TIMEOUT;
    }
    if (hc->err) {
      err = hc->err == 1 ? "traversal stack overflow" : "corrupt BVH (traversal bound exceeded)";
      return GR_E_INVALID;
    }
    return GR_OK;
  }
  cudaEvent_t ev[2];
  cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming);
  cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming);
  Counters* hc = f->ctr_host;
  long long it = 0;
  int batch = 0;
  gr_status status = GR_OK;
  for (;;) {
    for (int i = 0; i < B && e == cudaSuccess; ++i) e = launch();
    if (e != cudaSuccess) {
      err = std::string("launch: ") + cudaGetErrorString(e);
      status = GR_E_CUDA;
      break;
    }
    it += B;
    f->launches += (4LL + (hero ? 1 : 0)) * B;
    // copy the counters of this batch into pinned slot (batch & 1)
    e = cudaMemcpyAsync(hc + (batch & 1), f->ctr, sizeof(Counters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaEventRecord(ev[batch & 1], st);
    if (e != cudaSuccess) {
      err = std::string("counter copy: ") + cudaGetErrorString(e);
      status = GR_E_CUDA;
      break;
    }
    if (batch >= 1) {
      // wait for the previous batch while this one runs
      e = cudaEventSynchronize(ev[(batch - 1) & 1]);
      if (e != cudaSuccess) {
        err = std::string("event sync: ") + cudaGetErrorString(e);
        status = GR_E_CUDA;
        break;
      }
      const Counters& c = hc[(batch - 1) & 1];
      if (c.err) {
        err = c.err == 1 ? "traversal stack overflow" : "corrupt BVH (traversal bound exceeded)";
        status = GR_E_INVALID;
        break;
      }
      if (c.last_active == 0 && c.next_ticket >= c.total_tickets) break;
    }
    ++batch;
    if (it > max_iter) {
      err = "render exceeded its iteration bound";
      status = GR_E_TIMEOUT;
      break;
    }
  }
  f->iterations += it;
  if (profile) {
    // per-kernel device time of this render
    for (int k = 0; k < 4; ++k) {
      f->kernel_ms[k] = 0.0;
      f->kernel_launches[k] = 0;
    }
    if (status == GR_OK && !pev.empty()) cudaEventSynchronize(pev.back());
    // launch order regen, trace, shadow, shade; reported as 0 regen, 1 trace,
    // 2 shade, 3 shadow
    const int slot_of[4] = {0, 1, 3, 2};
    for (size_t i = 0; i + 4 < pev.size(); i += 5) {
      for (int k = 0; k < 4; ++k) {
        float ms = 0.0f;
        if (status == GR_OK && cudaEventElapsedTime(&ms, pev[i + k], pev[i + k + 1]) == cudaSuccess) {
          f->kernel_ms[slot_of[k]] += ms;
          f->kernel_launches[slot_of[k]] += 1;
        }
      }
    }
    for (auto e3 : pev) cudaEventDestroy(e3);
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  return status;
#undef GR_CK
}


// ================================================================== no-allocation variant
// gr_render_static runs the same four wavefront kernels, but its scratch (slot
// pool, queues, counters, view and table descriptors) lives in the fixed
// device array below instead of memory obtained from the CUDA allocator, and
// the accumulators are caller-owned device memory.  The array is part of the
// module image: every GPU that loads the library holds it until the process
// exits.  All calls share it, so calls that overlap on the GPU (two streams,
// two host threads) race on it; calls must be ordered.
static __device__ __align__(256) unsigned char g_static_scratch[GR_STATIC_SCRATCH_BYTES];

gr_status render_static_impl(gr_scene* const* scenes, int n_scenes, const gr_view_desc* vd, int n_views,
                             const gr_render_opts& o, float* accum, cudaStream_t st, std::string& err) {
  // The host-side name of the array is not a device address: ask the runtime
  // for it on every call, with the calling thread's device current (the
  // lookup allocates nothing, and a module reloaded after cudaDeviceReset
  // gets its new address).
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    return GR_E_CUDA;
  }
  void* sym = nullptr;
  e = cudaGetSymbolAddress(&sym, g_static_scratch);
  if (e != cudaSuccess || !sym) {
    err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
    return GR_E_CUDA;
  }
  unsigned char* base = (unsigned char*)sym;

  const int NSv = vd[0].n_stokes;
  const size_t tsize = o.table_dtype == GR_TABLE_F32 ? 4 : 2;
  std::vector<DevView> views;
  std::vector<DevScene> sc(n_scenes);
  std::vector<TableRow> rows;
  std::vector<TableBuildRow> brows;
  int vals = 0;
  unsigned long long total_tickets = 0;
  size_t acc_off = 0, acc_total = 0;
  for (int v = 0; v < n_views; ++v) acc_total += (size_t)vd[v].width * vd[v].height * vd[v].n_bins * vd[v].n_stokes;
  for (int i = 0; i < n_scenes; ++i) sc[i] = scenes[i]->dev;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = vd[v];
    DevView V;
    std::memset(&V, 0, sizeof V);
    V.W = d.width;
    V.H = d.height;
    V.nb = d.n_bins;
    V.ns = d.n_stokes;
    V.max_depth = d.max_depth;
    V.spp = d.spp;
    V.first_sample = d.first_sample;
    V.view_index = d.view_index;
    V.scene_index = d.scene_index;
    V.ortho = d.ortho;
    V.ortho_half = d.ortho_half_m;
    V.lmin = d.lambda_min_um;
    V.lmax = d.lambda_max_um;
    V.beta0 = d.f_beta * d.p_pix_um;
    V.ticket_base = (long long)total_tickets;
    V.Q = d.n_bins;  // no hero-wavelength MIS here
    V.hs = 1;
    V.nbu = std::min(d.spp, d.n_bins);
    V.n_tickets = (long long)V.nbu * d.width * d.height;
    total_tickets += (unsigned long long)V.n_tickets;
    V.acc_sum = accum + acc_off;
    V.acc_comp = accum + acc_total + acc_off;
    acc_off += (size_t)d.width * d.height * d.n_bins * d.n_stokes;
    const gr_scene* S = scenes[d.scene_index];
    V.table_base = (int)rows.size();
    for (size_t m = 0; m < S->mats.size(); ++m)
      for (int b = 0; b < d.n_bins; ++b) {
        TableRow r{0, -1};
        const gr_material& M = S->mats[m];
        if (M.type == GR_MAT_GRATING) {
          double lam = d.n_bins <= 1 ? (double)d.lambda_min_um
                                     : (double)d.lambda_min_um + (double)b * ((double)d.lambda_max_um - (double)d.lambda_min_um) /
                                                                     (double)(d.n_bins - 1);
          int jm = std::min(kMaxOrder, (int)std::floor(2.0 * (double)M.period_um / lam) + 2);
          r.offset = vals;
          r.jmax = jm;
          vals += jm + 1;
          TableBuildRow br{};
          br.offset = r.offset;
          br.jmax = jm;
          br.view = v;
          br.bin = b;
          br.height_um = M.height_um;
          brows.push_back(br);
        }
        rows.push_back(r);
      }
    views.push_back(V);
  }
  // --- carve the fixed array; anything that does not fit is rejected
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return r;
  };
  const size_t o_ctr = take(sizeof(Counters));
  const size_t o_views = take(sizeof(DevView) * n_views);
  const size_t o_vdesc = take(sizeof(gr_view_desc) * n_views);
  const size_t o_scenes = take(sizeof(DevScene) * n_scenes);
  const size_t o_rows = take(sizeof(TableRow) * rows.size());
  const size_t o_brows = take(sizeof(TableBuildRow) * brows.size());
  const size_t o_vals = take(tsize * (size_t)std::max(vals, 1));
  const size_t o_vals32 = o.table_dtype == GR_TABLE_F32 ? o_vals : take(sizeof(float) * (size_t)std::max(vals, 1));
  const size_t fixed = off;
  // the slot pool's 6 arrays each start on a 256-byte boundary: up to 6 x 255
  // bytes of padding, counted with the fixed part
  const size_t per_slot = sizeof(float4) * 14 + 2 * sizeof(float2) + sizeof(int4) + 2 * sizeof(int) + 1;
  const size_t slack = 7 * 256;
  const long long p_max = fixed + slack >= (size_t)GR_STATIC_SCRATCH_BYTES
                              ? 0
                              : (long long)(((size_t)GR_STATIC_SCRATCH_BYTES - fixed - slack) / per_slot) / 256 * 256;
  if (p_max < 256) {
    err = "views and order tables need " + std::to_string(fixed) + " bytes, which leaves fewer than 256 path slots "
          "in the static scratch of " + std::to_string((size_t)GR_STATIC_SCRATCH_BYTES) + " bytes";
    return GR_E_INVALID;
  }
  if (o.pool_size > p_max) {
    err = "pool_size " + std::to_string(o.pool_size) + " exceeds the static scratch capacity of " +
          std::to_string(p_max) + " slots";
    return GR_E_INVALID;
  }
  long long P = o.pool_size > 0 ? o.pool_size : p_max;
  P = std::min<long long>(P, (long long)std::max<unsigned long long>(total_tickets, 1ull));
  P = (P + 255) / 256 * 256;
  if (P > p_max) P = p_max;
  const size_t o_f4 = take(sizeof(float4) * (size_t)P * 14);
  const size_t o_hit = take(sizeof(float2) * (size_t)P * 2);  // hit, shh
  const size_t o_meta = take(sizeof(int4) * (size_t)P);
  const size_t o_tq = take(sizeof(int) * (size_t)P);
  const size_t o_sq = take(sizeof(int) * (size_t)P);
  const size_t o_st8 = take((size_t)P);
  if (off > (size_t)GR_STATIC_SCRATCH_BYTES) {
    err = "static scratch layout overflow";
    return GR_E_INVALID;
  }
  RenderParams p;
  std::memset(&p, 0, sizeof p);
  p.views = (const DevView*)(base + o_views);
  p.n_views = n_views;
  p.scenes = (const DevScene*)(base + o_scenes);
  p.seed = o.seed;
  p.flags = o.flags;
  p.rows = (const TableRow*)(base + o_rows);
  p.table_vals = base + o_vals;
  p.table_vals32 = (const float*)(base + o_vals32);
  p.table_dtype = o.table_dtype;
  p.table_rows = (int)rows.size();
  p.table_vals_count = vals;
  float4* f4 = (float4*)(base + o_f4);
  p.pool.od0 = f4;
  p.pool.od1 = f4 + (size_t)P;
  for (int r = 0; r < 4; ++r) p.pool.tp[r] = f4 + (size_t)P * (2 + r);
  p.pool.xf = f4 + (size_t)P * 6;
  p.pool.part = f4 + (size_t)P * 7;
  p.pool.accS = f4 + (size_t)P * 8;
  p.pool.accC = f4 + (size_t)P * 9;
  p.pool.shd = f4 + (size_t)P * 10;
  p.pool.shc = f4 + (size_t)P * 11;
  p.pool.shm = f4 + (size_t)P * 12;
  p.pool.mis = f4 + (size_t)P * 13;
  p.pool.hit = (float2*)(base + o_hit);
  p.pool.shh = p.pool.hit + (size_t)P;
  p.pool.meta = (int4*)(base + o_meta);
  p.pool.tq = (int*)(base + o_tq);
  p.pool.sq = (int*)(base + o_sq);
  p.pool.st8 = base + o_st8;
  p.P = (int)P;
  p.regen_thr = o.regen_threshold_pct;
  p.ctr = (Counters*)(base + o_ctr);
  const size_t smem_table = sizeof(TableRow) * rows.size() + tsize * vals;
  p.table_smem = smem_table <= 40 * 1024 ? 1 : 0;
  const size_t smem = p.table_smem ? align_up(smem_table, 16) : 0;
#define GR_SK(x)                                               \
  do {                                                         \
    e = (x);                                                   \
    if (e != cudaSuccess) {                                    \
      err = std::string(#x) + ": " + cudaGetErrorString(e);    \
      return GR_E_CUDA;                                        \
    }                                                          \
  } while (0)
  // the array keeps the previous call's contents: the counters and the slot
  // states (0 = idle) must start at zero
  Counters c0;
  std::memset(&c0, 0, sizeof c0);
  c0.total_tickets = total_tickets;
  GR_SK(cudaMemcpyAsync(base + o_ctr, &c0, sizeof c0, cudaMemcpyHostToDevice, st));
  GR_SK(cudaMemsetAsync(p.pool.meta, 0, sizeof(int4) * (size_t)P, st));
  GR_SK(cudaMemsetAsync(p.pool.st8, ST_IDLE, (size_t)P, st));
  GR_SK(cudaMemcpyAsync(base + o_views, views.data(), sizeof(DevView) * n_views, cudaMemcpyHostToDevice, st));
  GR_SK(cudaMemcpyAsync(base + o_vdesc, vd, sizeof(gr_view_desc) * n_views, cudaMemcpyHostToDevice, st));
  GR_SK(cudaMemcpyAsync(base + o_scenes, sc.data(), sizeof(DevScene) * n_scenes, cudaMemcpyHostToDevice, st));
  if (!rows.empty()) GR_SK(cudaMemcpyAsync(base + o_rows, rows.data(), sizeof(TableRow) * rows.size(), cudaMemcpyHostToDevice, st));
  k_views<<<(n_views + 63) / 64, 64, 0, st>>>((const gr_view_desc*)(base + o_vdesc), (DevView*)(base + o_views), n_views);
  if (!brows.empty()) {
    GR_SK(cudaMemcpyAsync(base + o_brows, brows.data(), sizeof(TableBuildRow) * brows.size(), cudaMemcpyHostToDevice, st));
    const TableBuildRow* br = (const TableBuildRow*)(base + o_brows);
    const int nr = (int)brows.size();
    if (o.table_dtype == GR_TABLE_F32)
      k_tables<float><<<nr, 64, 0, st>>>(br, nr, p.views, (float*)(base + o_vals), nullptr);
    else if (o.table_dtype == GR_TABLE_F16)
      k_tables<__half><<<nr, 64, 0, st>>>(br, nr, p.views, (__half*)(base + o_vals), (float*)(base + o_vals32));
    else
      k_tables<__nv_bfloat16><<<nr, 64, 0, st>>>(br, nr, p.views, (__nv_bfloat16*)(base + o_vals), (float*)(base + o_vals32));
  }
  GR_SK(cudaGetLastError());
  // --- launch shapes (same rule as gr_render)
  const int sms = sm_count(dev);
  const int block = o.block > 0 ? o.block : 256;
  auto grid_for = [&](const void* fn, size_t dyn, int blk = 0) {
    int per = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, blk > 0 ? blk : block, dyn);
    return sms * std::max(per, 1);
  };
  const void* shade_fn = shade_kernel(NSv, o.table_dtype, 0);
  const int gmax = (int)((P + block - 1) / block);
  const int g_regen = std::min((int)((P + (long long)block * GR_REGEN_SLOTS - 1) / ((long long)block * GR_REGEN_SLOTS)),
                               grid_for(regen_kernel(NSv, false), 0));
  const int tree = pick_tree(o.flags, scenes, n_scenes);
  const int tblk = tree == kTreeWide ? block : trace_block(block);
  const int g_trace = std::min((int)((P + tblk - 1) / tblk), grid_for(trace_kernel(tree), 0, tblk));
  const int g_shade = std::min(gmax, grid_for(shade_fn, smem));
  const int g_shadow = shadow_grid(P, sms);
  // --- iteration loop; the host reads the device counters into a stack copy
  // after every batch (no events, no pinned buffer)
  long long n_max = 1, d_max = 0;
  for (int v = 0; v < n_views; ++v) {
    n_max = std::max<long long>(n_max, (long long)vd[v].spp / vd[v].n_bins + 1);
    d_max = std::max<long long>(d_max, vd[v].max_depth);
  }
  const int B = 8;
  const long long worst = ((long long)((total_tickets + P - 1) / P) + 1) * n_max * (d_max + 3) + 4 * B;
  const long long max_iter = o.max_iterations > 0 ? o.max_iterations : 2 * worst;
  long long it = 0;
  for (;;) {
    for (int i = 0; i < B; ++i) {
      if (NSv == 1) {
        if (o.table_dtype == GR_TABLE_F32) e = launch_iteration<1, float>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, nullptr);
        else if (o.table_dtype == GR_TABLE_F16) e = launch_iteration<1, __half>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, nullptr);
        else e = launch_iteration<1, __nv_bfloat16>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, nullptr);
      } else {
        if (o.table_dtype == GR_TABLE_F32) e = launch_iteration<4, float>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, nullptr);
        else if (o.table_dtype == GR_TABLE_F16) e = launch_iteration<4, __half>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, nullptr);
        else e = launch_iteration<4, __nv_bfloat16>(p, tree, g_regen, g_trace, g_shade, g_shadow, block, smem, st, nullptr);
      }
      if (e != cudaSuccess) {
        err = std::string("launch: ") + cudaGetErrorString(e);
        return GR_E_CUDA;
      }
    }
    it += B;
    Counters hc;
    GR_SK(cudaMemcpyAsync(&hc, base + o_ctr, sizeof hc, cudaMemcpyDeviceToHost, st));
    GR_SK(cudaStreamSynchronize(st));
    if (hc.err) {
      err = hc.err == 1 ? "traversal stack overflow" : "corrupt BVH (traversal bound exceeded)";
      return GR_E_INVALID;
    }
    if (hc.last_active == 0 && hc.next_ticket >= hc.total_tickets) break;
    if (it > max_iter) {
      err = "render exceeded its iteration bound";
      return GR_E_TIMEOUT;
    }
  }
#undef GR_SK
  return GR_OK;
}

cudaError_t readback_impl(gr_frame* f, int v, float* dst_dev, const float* inv_count_dev, cudaStream_t st) {
  const gr_view_shape& s = f->shapes[v];
  const long long n = (long long)s.W * s.H * s.nb * s.ns;
  int blocks = (int)std::min<long long>((n + 255) / 256, 65535);
  k_readback<<<blocks, 256, 0, st>>>(f->acc + f->offsets[v], f->acc + f->acc_floats + f->offsets[v], s.W, s.H, s.nb,
                                      s.ns, inv_count_dev, dst_dev);
  return cudaGetLastError();
}

}  // namespace gr
