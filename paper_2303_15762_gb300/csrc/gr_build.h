// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "gr.h"
#include "gr_device.cuh"

namespace gr {

cudaError_t build_lbvh(const float* verts, const int* tri_mat, int n, float4* tri, int* tmat, float* nodes,
                       unsigned long long* keys_out, cudaStream_t st);
cudaError_t build_wide(const float* nodes, const float4* tri, int n, uint4* wn, int* n_wide, cudaStream_t st);
cudaError_t build_half(const float* nodes, int n, uint4* hn, cudaStream_t st);

// Largest slot pool (the trace launch tags next-event entries with bit 30 of
// the slot index).
constexpr int kMaxPool = (1 << 30) - 256;

// Wavefront slot pool: per-slot path state in structure-of-arrays form.
struct Pool {
  float4* od0;   // o.xyz, beta^2 (um^2)
  float4* od1;   // d.xyz, rho
  float4* tp[4]; // throughput: scalar in tp[0].x, or Mueller rows 0..3
  float4* xf;    // Stokes frame x axis (w unused)
  float4* part;  // contribution of the current sample
  float4* accS;  // ticket sums (Kahan)
  float4* accC;  // ticket compensations
  float4* shd;   // NEE direction xyz, (emitter index | vertex segment << 16)
  float4* shc;   // NEE throughput column (Stokes vector)
  float4* shm;   // NEE lobe terms: squared offset, g, (k l)^2, cos
  float4* mis;   // lobe terms of the vertex that sampled the current direction
  float2* hit;   // t, leaf slot
  float2* shh;   // the next-event ray's closest hit: t, leaf slot
  int4* meta;    // view, local ticket, (sample k | seg << 16 | state << 24 | delta << 26), previous leaf slot
  int* tq;       // trace queue
  int* sq;       // shadow queue
  unsigned char* st8;  // slot state (idle / active / done / waiting): the one field k_regen scans for every slot
  // hero-wavelength MIS only (null otherwise); planes [g * P + slot] for the
  // class member g (bin c + g Q)
  float4* hq;    // path density ratios q_g of the class wavelengths to the hero's
  float4* hqp;   // the same ratios before the latest interaction
  float4* haccS; // [4] ticket sums of member g (Kahan)
  float4* haccC; // [4] ticket compensations of member g
  int* dq;       // the density queue (slots whose ratios k_density completes)
  float* hsub;   // per class record (views with hs > 1): [range][member][Stokes] totals
  int* hsub_n;   // per class record: ranges folded so far (the last one adds all)
  // anisotropic footprints only (null otherwise): K = Kr + i Ki in the ray's
  // frame (xf), as (Kr11, Kr12, Kr22, Ki11), (Ki12, Ki22, -, -); the same for
  // a next-event request in the frame nkf of its direction
  float4* ak0;
  float4* ak1;
  float4* nk0;
  float4* nk1;
  float4* nkf;
};

struct Counters {
  unsigned long long next_ticket;
  unsigned long long total_tickets;
  int tq_count;  // trace-queue entries filled from the front (continuing segments)
  int sq_count;
  int last_active;
  int err;
  int trace_next;  // next unclaimed trace-queue entry (claimed in groups of 32)
  int tq_back;     // trace-queue entries filled from the end of the array (camera rays)
  int dq_count;    // hero-wavelength MIS: rough vertices queued for k_density
  int sq_done;     // k_shadow blocks finished (the last one closes the queues)
  int tq_front, tq_n;  // the iteration's trace queue as k_shade reads it
  unsigned long long samples, segments, shadow, ref_hit, ref_lobe, iters, node_visits, tri_tests;
  unsigned long long held;  // finished samples k_regen held back for their next-event ray
};

struct RenderParams {
  const DevView* views;
  int n_views;
  const DevScene* scenes;
  uint32_t seed;
  int flags;
  const TableRow* rows;
  const void* table_vals;
  const float* table_vals32;  // the same values in FP32 (== table_vals for FP32 tables)
  int table_dtype;
  int table_smem;        // 1 if the order table is staged in shared memory
  int table_rows;
  int table_vals_count;
  Pool pool;
  int P;
  int regen_thr;         // regeneration threshold, percent of idle slots (0 = always)
  Counters* ctr;
};

// FP32 FMA microbenchmark (gr_peak.cu): TFLOP/s and the best launch's ms.
cudaError_t fma_peak_impl(cudaStream_t st, double* tflops, double* best_ms);

// Inspection helpers (gr_render.cu): one order-table row decoded to float
// [jmax + 1]; the footprint update of n (beta^2, rho, t, kw) quadruples.
cudaError_t debug_table_impl(float height_um, double lambda_um, int jmax, int dtype, float* host_out,
                             cudaStream_t st);
cudaError_t debug_footprint_impl(int n, const float* host_in, float* host_out, cudaStream_t st);

// Footprint-resolved generalized rays through a 1D aperture (gr_aperture.cu).
cudaError_t aperture_backward_impl(int n_det, const double* x0_host, int n_ap, const double* xa_host,
                                   const double* wa_host, double beta, double z, double k, double reach,
                                   double dtheta, double rho_cut, double* out_host, cudaStream_t st, float* ms);
cudaError_t aperture_backward_3d_impl(int n_det, const double* x0_host, int n_ap, const double* xa_host,
                                      const double* wa_host, double beta, double z, double k, double reach,
                                      double dt, double rho_cut, double* out_host, cudaStream_t st, float* ms);

}  // namespace gr

struct gr_scene {
  gr::DevScene dev;
  void* mem = nullptr;            // single device allocation holding every array
  unsigned long long* keys = nullptr;
  int n_tris = 0;
  std::vector<gr_material> mats;  // host copy (order tables)
  int device = 0;
  size_t bytes = 0;               // size of `mem`
};

struct gr_view_shape {
  int W, H, nb, ns;
};

struct gr_frame {
  int n_views = 0;
  std::vector<gr_view_shape> shapes;
  std::vector<size_t> offsets;           // float offset of each view's sum plane
  float* acc = nullptr;                  // sums then compensations
  bool owns_acc = true;                  // false: caller-owned device buffer (gr_frame_wrap)
  size_t acc_floats = 0;                 // floats per plane set (sum part)
  std::vector<std::vector<long long>> counts;  // [view][bin] samples accumulated
  // scratch kept between renders
  void* scratch = nullptr;
  size_t scratch_bytes = 0;
  gr::Counters* ctr = nullptr;           // device counters
  gr::Counters* ctr_host = nullptr;      // pinned mirror
  long long launches = 0;
  long long iterations = 0;
  // cached single-launch render graph and the launch parameters it was built for
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;   // private stream used only to record the graph
  std::vector<unsigned char> graph_key;
  double kernel_ms[4] = {0, 0, 0, 0};       // last profiled render: regen, trace, shade, shadow
  long long kernel_launches[4] = {0, 0, 0, 0};
  int device = 0;
};
