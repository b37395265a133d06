// C ABI entry points of libgr.so (declared and documented in include/gr.h).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "gr_build.h"
#include "gr_measure.h"

namespace gr {
gr_status render_impl(gr_scene* const* scenes, int n_scenes, const gr_view_desc* vd, int n_views,
                      const gr_render_opts& o, gr_frame* f, const std::vector<float*>& acc_sum,
                      const std::vector<float*>& acc_comp, cudaStream_t st, std::string& err,
                      size_t* plan_bytes = nullptr);
cudaError_t readback_impl(gr_frame* f, int v, float* dst_dev, const float* inv_count_dev, cudaStream_t st);
cudaError_t debug_rng_impl(uint32_t seed, uint32_t view, uint32_t pixel, uint32_t sample, int seg, int call, int n,
                           uint32_t* host_out, cudaStream_t st);
gr_status render_static_impl(gr_scene* const* scenes, int n_scenes, const gr_view_desc* vd, int n_views,
                             const gr_render_opts& o, float* accum, cudaStream_t st, std::string& err);
}  // namespace gr

namespace {

thread_local std::string g_err = "no error";

gr_status fail(gr_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

gr_status cuda_fail(cudaError_t e, const char* what) {
  return fail(e == cudaErrorMemoryAllocation ? GR_E_OOM : GR_E_CUDA,
              std::string(what) + ": " + cudaGetErrorString(e));
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Every scene of a render must live on the calling thread's current device
// (its BVH and triangles are read by kernels launched there).
gr_status check_scene_devices(const std::string& who, gr_scene* const* scenes, int n_scenes, int dev) {
  for (int i = 0; i < n_scenes; ++i)
    if (scenes[i]->device != dev)
      return fail(GR_E_INVALID, who + ": scene " + std::to_string(i) + " was created on device " +
                                    std::to_string(scenes[i]->device) + ", the current device is " +
                                    std::to_string(dev));
  return GR_OK;
}

// A caller-owned accumulator buffer must be device (or managed) memory that
// the current device owns; a host pointer would fault in the kernels.
gr_status check_device_buffer(const std::string& who, const void* p, int dev) {
  cudaPointerAttributes a;
  const cudaError_t e = cudaPointerGetAttributes(&a, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(GR_E_INVALID, who + ": accumulator pointer is not known to CUDA (" + cudaGetErrorString(e) + ")");
  }
  if (!((a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev))
    return fail(GR_E_INVALID, who + ": accumulators must be device memory of the current device " +
                                  std::to_string(dev));
  return GR_OK;
}

int current_device() {
  int d = -1;
  if (cudaGetDevice(&d) != cudaSuccess) return -1;
  return d;
}

// Frame over caller-owned accumulators (acc != nullptr, not zeroed: the
// caller's buffer is added into) or library-owned ones (zeroed on stream).
gr_status frame_make(const char* who, const gr_view_desc* views, int32_t n_views, float* acc, cudaStream_t st,
                     gr_frame** out) {
  const std::string w(who);
  if (!views || !out || n_views <= 0) return fail(GR_E_INVALID, w + ": bad arguments");
  size_t total = 0;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = views[v];
    if (d.width <= 0 || d.height <= 0 || d.n_bins <= 0 || d.n_bins > 4096 || (d.n_stokes != 1 && d.n_stokes != 4))
      return fail(GR_E_INVALID, w + ": bad view shape " + std::to_string(v));
    if ((long long)d.width * d.height * d.n_bins >= (1LL << 31))
      return fail(GR_E_INVALID, w + ": view too large " + std::to_string(v));
    total += (size_t)d.width * d.height * d.n_bins * d.n_stokes;
  }
  const int dev = current_device();
  if (dev < 0) return fail(GR_E_CUDA, w + ": no current CUDA device");
  if (acc) {
    const gr_status s = check_device_buffer(w, acc, dev);
    if (s != GR_OK) return s;
  }
  gr_frame* F = new (std::nothrow) gr_frame();
  if (!F) return fail(GR_E_OOM, w + ": host allocation");
  F->device = dev;
  F->n_views = n_views;
  size_t off = 0;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = views[v];
    F->shapes.push_back(gr_view_shape{d.width, d.height, d.n_bins, d.n_stokes});
    F->offsets.push_back(off);
    off += (size_t)d.width * d.height * d.n_bins * d.n_stokes;
    F->counts.emplace_back(d.n_bins, 0LL);
  }
  F->acc_floats = total;
  F->owns_acc = acc == nullptr;
  cudaError_t e = cudaSuccess;
  if (acc) {
    F->acc = acc;
  } else {
    e = cudaMallocAsync(&F->acc, sizeof(float) * total * 2, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(F->acc, 0, sizeof(float) * total * 2, st);
  }
  if (e == cudaSuccess) e = cudaMallocAsync(&F->ctr, sizeof(gr::Counters), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(F->ctr, 0, sizeof(gr::Counters), st);
  if (e == cudaSuccess) e = cudaHostAlloc(&F->ctr_host, sizeof(gr::Counters) * 2, cudaHostAllocDefault);
  if (e != cudaSuccess) {
    if (F->acc && F->owns_acc) cudaFreeAsync(F->acc, st);
    if (F->ctr) cudaFreeAsync(F->ctr, st);
    delete F;
    return cuda_fail(e, w.c_str());
  }
  std::memset(F->ctr_host, 0, sizeof(gr::Counters) * 2);
  *out = F;
  return GR_OK;
}

}  // namespace

extern "C" {

int32_t gr_abi_version(void) { return 1; }

gr_status gr_measure_fp32_peak(void* cuda_stream, double* tflops_out, double* ms_out) {
  if (!tflops_out || !ms_out) return fail(GR_E_INVALID, "gr_measure_fp32_peak: null argument");
  double tf = 0.0, ms = 0.0;
  const cudaError_t e = gr::fma_peak_impl((cudaStream_t)cuda_stream, &tf, &ms);
  if (e != cudaSuccess) return cuda_fail(e, "gr_measure_fp32_peak");
  *tflops_out = tf;
  *ms_out = ms;
  return GR_OK;
}

const char* gr_last_error(void) { return g_err.c_str(); }

gr_status gr_scene_create(const gr_scene_desc* desc, void* cuda_stream, gr_scene** out) {
  if (!desc || !out) return fail(GR_E_INVALID, "gr_scene_create: null argument");
  const int n = desc->n_tris;
  if (n < 0 || desc->n_mats < 0 || desc->n_lights < 0) return fail(GR_E_INVALID, "gr_scene_create: negative count");
  if (n > 0 && (!desc->verts || !desc->tri_mat)) return fail(GR_E_INVALID, "gr_scene_create: null triangle arrays");
  if (desc->n_mats > 0 && !desc->mats) return fail(GR_E_INVALID, "gr_scene_create: null materials");
  if (desc->n_lights > 0 && !desc->lights) return fail(GR_E_INVALID, "gr_scene_create: null lights");
  if (n > (1 << 28)) return fail(GR_E_INVALID, "gr_scene_create: too many triangles");
  for (int i = 0; i < desc->n_mats; ++i) {
    const gr_material& M = desc->mats[i];
    if (M.type < GR_MAT_ABSORBER || M.type > GR_MAT_DIELECTRIC || M.fresnel < 0 || M.fresnel > 1)
      return fail(GR_E_INVALID, "gr_scene_create: bad material " + std::to_string(i));
    if (M.type == GR_MAT_GRATING && !(M.period_um > 0.0f))
      return fail(GR_E_INVALID, "gr_scene_create: grating period must be > 0");
    if (M.type == GR_MAT_ROUGH && !(M.corr_len_um > 0.0f))
      return fail(GR_E_INVALID, "gr_scene_create: correlation length must be > 0");
    if (M.type == GR_MAT_DIELECTRIC && !(M.n_re > 0.0f && M.cauchy_b_um2 >= 0.0f))
      return fail(GR_E_INVALID, "gr_scene_create: dielectric index must be > 0 (n_re > 0, cauchy_b_um2 >= 0)");
  }
  for (int i = 0; i < desc->n_lights; ++i) {
    const gr_light& L = desc->lights[i];
    if (L.type != GR_LIGHT_DISTANT && L.type != GR_LIGHT_ENV)
      return fail(GR_E_INVALID, "gr_scene_create: bad light " + std::to_string(i));
  }
  for (int i = 0; i < n; ++i)
    if (desc->tri_mat[i] < 0 || desc->tri_mat[i] >= desc->n_mats)
      return fail(GR_E_INVALID, "gr_scene_create: material index out of range at triangle " + std::to_string(i));

  cudaStream_t st = (cudaStream_t)cuda_stream;
  gr_scene* S = new (std::nothrow) gr_scene();
  if (!S) return fail(GR_E_OOM, "gr_scene_create: host allocation");
  cudaGetDevice(&S->device);
  S->n_tris = n;
  S->mats.assign(desc->mats, desc->mats + desc->n_mats);

  // emitters: triangles grouped by emitter material (host bookkeeping)
  std::vector<int> emitter_of_mat(std::max(desc->n_mats, 1), -1);
  std::vector<std::vector<int>> groups;
  for (int i = 0; i < n; ++i) {
    int m = desc->tri_mat[i];
    if (desc->mats[m].type != GR_MAT_EMITTER) continue;
    if (emitter_of_mat[m] < 0) {
      emitter_of_mat[m] = (int)groups.size();
      groups.emplace_back();
    }
    groups[emitter_of_mat[m]].push_back(i);
  }
  std::vector<gr::DevEmitter> emit;
  std::vector<float4> etris;
  for (size_t g = 0; g < groups.size(); ++g) {
    gr::DevEmitter E;
    std::memset(&E, 0, sizeof E);
    E.mat = desc->tri_mat[groups[g][0]];
    E.first = (int)(etris.size() / 3);
    E.count = (int)groups[g].size();
    for (int a = 0; a < 3; ++a) {
      E.lo[a] = 3.4e38f;
      E.hi[a] = -3.4e38f;
    }
    for (int t : groups[g])
      for (int k = 0; k < 3; ++k) {
        const float* v = desc->verts + 9 * t + 3 * k;
        etris.push_back(make_float4(v[0], v[1], v[2], 0.0f));
        for (int a = 0; a < 3; ++a) {
          E.lo[a] = std::min(E.lo[a], v[a]);
          E.hi[a] = std::max(E.hi[a], v[a]);
        }
      }
    // planar when every vertex lies within 1e-6 of the extent from the first
    // triangle's plane (the next-event precheck relies on it)
    {
      const float* v0 = desc->verts + 9 * groups[g][0];
      const double e1[3] = {(double)v0[3] - v0[0], (double)v0[4] - v0[1], (double)v0[5] - v0[2]};
      const double e2[3] = {(double)v0[6] - v0[0], (double)v0[7] - v0[1], (double)v0[8] - v0[2]};
      double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
      const double ln = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      double ext = 0.0;
      for (int a = 0; a < 3; ++a) ext = std::max(ext, (double)E.hi[a] - E.lo[a]);
      bool planar = ln > 0.0;
      for (int t : groups[g])
        for (int k = 0; k < 3 && planar; ++k) {
          const float* v = desc->verts + 9 * t + 3 * k;
          const double dist = ((v[0] - (double)v0[0]) * n[0] + (v[1] - (double)v0[1]) * n[1] +
                               (v[2] - (double)v0[2]) * n[2]) / ln;
          planar = std::fabs(dist) <= 1e-6 * ext;
        }
      E.planar = planar ? 1 : 0;
      // the unit normal, once per scene (FP64, and rounded to FP32)
      for (int a = 0; a < 3; ++a) {
        E.nd[a] = n[a] / ln;
        E.n[a] = (float)E.nd[a];
      }
    }
    emit.push_back(E);
  }

  // one device allocation for every persistent array
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t r = off;
    off = align_up(off + std::max<size_t>(bytes, 1), 256);
    return r;
  };
  const size_t o_tri = take(sizeof(float4) * 3 * (size_t)n);
  const size_t o_tmat = take(sizeof(int) * (size_t)n);
  const size_t o_nodes = take(sizeof(float) * 16 * (size_t)std::max(n - 1, 0));
  const size_t o_mats = take(sizeof(gr_material) * desc->n_mats);
  const size_t o_lights = take(sizeof(gr_light) * desc->n_lights);
  const size_t o_emit = take(sizeof(gr::DevEmitter) * emit.size());
  const size_t o_eom = take(sizeof(int) * emitter_of_mat.size());
  const size_t o_etri = take(sizeof(float4) * etris.size());
  const size_t o_keys = take(sizeof(unsigned long long) * (size_t)n);
  const size_t o_wide = take(sizeof(uint4) * 4 * (size_t)std::max(n - 1, 1));
  // FP16 nodes only when every coordinate is within +-16384 (finite boxes)
  bool half_ok = n >= 2;
  for (size_t i = 0; half_ok && i < 9 * (size_t)n; ++i) half_ok = std::fabs(desc->verts[i]) <= 16384.0f;
  const size_t o_half = take(half_ok ? sizeof(uint4) * 2 * (size_t)(n - 1) : 0);
  int n_wide = 0;
  cudaError_t e = cudaMallocAsync(&S->mem, off, st);
  if (e != cudaSuccess) {
    delete S;
    return cuda_fail(e, "gr_scene_create: device allocation");
  }
  unsigned char* b = (unsigned char*)S->mem;
  float* verts_d = nullptr;
  int* tmat_in = nullptr;
  gr_status status = GR_OK;
  do {
    if (n > 0) {
      if ((e = cudaMallocAsync(&verts_d, sizeof(float) * 9 * (size_t)n, st)) != cudaSuccess) break;
      if ((e = cudaMallocAsync(&tmat_in, sizeof(int) * (size_t)n, st)) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(verts_d, desc->verts, sizeof(float) * 9 * (size_t)n, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
      if ((e = cudaMemcpyAsync(tmat_in, desc->tri_mat, sizeof(int) * (size_t)n, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    }
    if (desc->n_mats && (e = cudaMemcpyAsync(b + o_mats, desc->mats, sizeof(gr_material) * desc->n_mats, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if (desc->n_lights && (e = cudaMemcpyAsync(b + o_lights, desc->lights, sizeof(gr_light) * desc->n_lights, cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if (!emit.empty() && (e = cudaMemcpyAsync(b + o_emit, emit.data(), sizeof(gr::DevEmitter) * emit.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if ((e = cudaMemcpyAsync(b + o_eom, emitter_of_mat.data(), sizeof(int) * emitter_of_mat.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if (!etris.empty() && (e = cudaMemcpyAsync(b + o_etri, etris.data(), sizeof(float4) * etris.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) break;
    if (n > 0) {
      e = gr::build_lbvh(verts_d, tmat_in, n, (float4*)(b + o_tri), (int*)(b + o_tmat), (float*)(b + o_nodes),
                         (unsigned long long*)(b + o_keys), st);
      if (e != cudaSuccess) break;
      e = gr::build_wide((const float*)(b + o_nodes), (const float4*)(b + o_tri), n, (uint4*)(b + o_wide), &n_wide, st);
      if (e != cudaSuccess) break;
      if (half_ok && (e = gr::build_half((const float*)(b + o_nodes), n, (uint4*)(b + o_half), st)) != cudaSuccess)
        break;
    }
    // host arrays are pageable: make sure every copy has consumed them
    e = cudaStreamSynchronize(st);
  } while (0);
  if (verts_d) cudaFreeAsync(verts_d, st);
  if (tmat_in) cudaFreeAsync(tmat_in, st);
  if (e != cudaSuccess) {
    status = cuda_fail(e, "gr_scene_create");
    cudaFreeAsync(S->mem, st);
    delete S;
    return status;
  }
  gr::DevScene& D = S->dev;
  D.n_tris = n;
  D.n_mats = desc->n_mats;
  D.n_lights = desc->n_lights;
  D.n_emitters = (int)emit.size();
  D.tri = (const float4*)(b + o_tri);
  D.tri_mat = (const int*)(b + o_tmat);
  D.nodes = (const float4*)(b + o_nodes);
  D.wnodes = (const uint4*)(b + o_wide);
  D.hnodes = half_ok ? (const uint4*)(b + o_half) : nullptr;
  D.n_wide = n_wide;
  D.pad_w = 0;
  D.mats = (const gr_material*)(b + o_mats);
  D.lights = (const gr_light*)(b + o_lights);
  D.emitters = (const gr::DevEmitter*)(b + o_emit);
  D.emitter_of_mat = (const int*)(b + o_eom);
  D.emitter_tris = (const float4*)(b + o_etri);
  S->keys = (unsigned long long*)(b + o_keys);
  S->bytes = off;
  *out = S;
  return GR_OK;
}

gr_status gr_scene_bytes(const gr_scene* scene, size_t* bytes_out) {
  if (!scene || !bytes_out) return fail(GR_E_INVALID, "gr_scene_bytes: null argument");
  *bytes_out = scene->bytes;
  return GR_OK;
}

gr_status gr_scene_destroy(gr_scene* scene) {
  if (!scene) return fail(GR_E_INVALID, "gr_scene_destroy: null scene");
  if (scene->mem) cudaFree(scene->mem);
  delete scene;
  return GR_OK;
}

gr_status gr_scene_bvh(gr_scene* scene, int32_t* n_out, uint64_t* keys, int32_t* children, float* boxes) {
  if (!scene || !n_out) return fail(GR_E_INVALID, "gr_scene_bvh: null argument");
  const int n = scene->n_tris;
  *n_out = n;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_fail(e, "gr_scene_bvh");
  if (keys && n > 0) {
    e = cudaMemcpy(keys, scene->keys, sizeof(uint64_t) * n, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "gr_scene_bvh keys");
  }
  if ((children || boxes) && n > 1) {
    std::vector<float> nodes((size_t)16 * (n - 1));
    e = cudaMemcpy(nodes.data(), scene->dev.nodes, sizeof(float) * nodes.size(), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "gr_scene_bvh nodes");
    for (int i = 0; i < n - 1; ++i) {
      if (children) {
        std::memcpy(children + 2 * i, &nodes[16 * (size_t)i + 12], 8);
      }
      if (boxes) std::memcpy(boxes + 12 * (size_t)i, &nodes[16 * (size_t)i], 48);
    }
  }
  return GR_OK;
}

gr_status gr_frame_create(const gr_view_desc* views, int32_t n_views, void* cuda_stream, gr_frame** out) {
  return frame_make("gr_frame_create", views, n_views, nullptr, (cudaStream_t)cuda_stream, out);
}

gr_status gr_frame_wrap(const gr_view_desc* views, int32_t n_views, float* accum_device, void* cuda_stream,
                        gr_frame** out) {
  return frame_make("gr_frame_wrap", views, n_views, accum_device, (cudaStream_t)cuda_stream, out);
}

gr_status gr_frame_bytes(const gr_frame* f, size_t* bytes_out) {
  if (!f || !bytes_out) return fail(GR_E_INVALID, "gr_frame_bytes: null argument");
  *bytes_out = (f->owns_acc ? sizeof(float) * f->acc_floats * 2 : 0) + sizeof(gr::Counters) + f->scratch_bytes;
  return GR_OK;
}

gr_status gr_frame_reset(gr_frame* f, void* cuda_stream) {
  if (!f) return fail(GR_E_INVALID, "gr_frame_reset: null frame");
  cudaError_t e = cudaMemsetAsync(f->acc, 0, sizeof(float) * f->acc_floats * 2, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_frame_reset");
  for (auto& c : f->counts) std::fill(c.begin(), c.end(), 0LL);
  return GR_OK;
}

gr_status gr_frame_release(gr_frame* f) {
  if (!f) return fail(GR_E_INVALID, "gr_frame_release: null frame");
  cudaDeviceSynchronize();
  if (f->acc && f->owns_acc) cudaFree(f->acc);
  if (f->scratch) cudaFree(f->scratch);
  if (f->ctr) cudaFree(f->ctr);
  if (f->ctr_host) cudaFreeHost(f->ctr_host);
  if (f->graph_exec) cudaGraphExecDestroy(f->graph_exec);
  if (f->capture_stream) cudaStreamDestroy(f->capture_stream);
  delete f;
  return GR_OK;
}

namespace {

// Checks shared by gr_render and gr_render_multi: options, scene indices,
// sample ranges, spectral and camera parameters, and the frame view each view
// accumulates into.
gr_status check_render_args(const char* who, gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views,
                            int32_t n_views, const gr_render_opts* opts, gr_frame* const* frames,
                            const int32_t* frame_view) {
  const std::string w(who);
  if (!scenes || !views || !opts || !frames || n_views <= 0 || n_scenes <= 0)
    return fail(GR_E_INVALID, w + ": null or empty argument");
  for (int i = 0; i < n_scenes; ++i)
    if (!scenes[i]) return fail(GR_E_INVALID, w + ": null scene " + std::to_string(i));
  if (opts->table_dtype < GR_TABLE_F32 || opts->table_dtype > GR_TABLE_BF16)
    return fail(GR_E_INVALID, w + ": bad table dtype");
  if (opts->pool_size < 0 || opts->pool_size > gr::kMaxPool || opts->block < 0 ||
      (opts->block && (opts->block % 32 || opts->block > 256)))
    return fail(GR_E_INVALID, w + ": bad pool size (0 to 2^30 - 256) or block (a multiple of 32, <= 256)");
  if (opts->regen_threshold_pct < 0 || opts->regen_threshold_pct > 100)
    return fail(GR_E_INVALID, w + ": regen_threshold_pct out of [0, 100]");
  const int ns = views[0].n_stokes;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = views[v];
    const gr_frame* fr = frames[v];
    const int fv = frame_view ? frame_view[v] : v;
    if (!fr || fv < 0 || fv >= fr->n_views)
      return fail(GR_E_INVALID, w + ": view " + std::to_string(v) + " has no frame view");
    const gr_view_shape& s = fr->shapes[fv];
    if (d.width != s.W || d.height != s.H || d.n_bins != s.nb || d.n_stokes != s.ns)
      return fail(GR_E_INVALID, w + ": view " + std::to_string(v) + " does not match its frame view");
    if (d.n_stokes != ns) return fail(GR_E_INVALID, w + ": all views of one call need the same n_stokes");
    if (d.scene_index < 0 || d.scene_index >= n_scenes)
      return fail(GR_E_INVALID, w + ": scene index out of range in view " + std::to_string(v));
    if (d.spp < 0 || d.first_sample < 0 || (long long)d.first_sample + d.spp >= (1LL << 31))
      return fail(GR_E_INVALID, w + ": bad sample range in view " + std::to_string(v));
    if ((long long)d.spp / d.n_bins + 1 >= 65536)
      return fail(GR_E_INVALID, w + ": more than 65535 samples per pixel and bin in one call");
    if ((opts->flags & GR_FLAG_HERO) && (opts->flags & GR_FLAG_ANISO))
      return fail(GR_E_INVALID, w + ": GR_FLAG_HERO and GR_FLAG_ANISO are not combined");
    if (opts->flags & GR_FLAG_HERO) {
      if (d.n_bins % 4 != 0)
        return fail(GR_E_INVALID, w + ": hero-wavelength MIS needs n_bins to be a multiple of 4 (view " +
                                      std::to_string(v) + ")");
      if ((long long)d.spp / (d.n_bins / 4) + 1 >= 65536)
        return fail(GR_E_INVALID, w + ": more than 65535 samples per pixel and class of 4 bins in one call");
    }
    if (d.max_depth < 0 || d.max_depth > 250) return fail(GR_E_INVALID, w + ": max_depth out of [0, 250]");
    if (!(d.lambda_min_um > 0.0f) || d.lambda_max_um < d.lambda_min_um || !(d.p_pix_um > 0.0f) || !(d.f_beta > 0.0f))
      return fail(GR_E_INVALID, w + ": bad spectral range or pixel footprint in view " + std::to_string(v));
    if (!(d.vfov_deg > 0.0f && d.vfov_deg < 180.0f) && !d.ortho)
      return fail(GR_E_INVALID, w + ": bad field of view in view " + std::to_string(v));
  }
  // two views must not accumulate into the same frame view in one call
  for (int a = 0; a < n_views; ++a)
    for (int b = a + 1; b < n_views && n_views <= 4096; ++b)
      if (frames[a] == frames[b] && (frame_view ? frame_view[a] == frame_view[b] : a == b))
        return fail(GR_E_INVALID, w + ": two views accumulate into the same frame view");
  return GR_OK;
}

// Scenes and frames of one render must all belong to the current device.
gr_status check_call_devices(const char* who, gr_scene* const* scenes, int32_t n_scenes, gr_frame* const* frames,
                             int32_t n_frames) {
  const std::string w(who);
  const int dev = current_device();
  if (dev < 0) return fail(GR_E_CUDA, w + ": no current CUDA device");
  gr_status s = check_scene_devices(w, scenes, n_scenes, dev);
  if (s != GR_OK) return s;
  for (int i = 0; i < n_frames; ++i)
    if (frames[i]->device != dev)
      return fail(GR_E_INVALID, w + ": frame of view " + std::to_string(i) + " was created on device " +
                                    std::to_string(frames[i]->device) + ", the current device is " +
                                    std::to_string(dev));
  return GR_OK;
}

void add_counts(gr_frame* fr, int fv, const gr_view_desc& d) {
  for (int b = 0; b < d.n_bins; ++b) {
    long long r = ((long long)b - d.first_sample) % d.n_bins;
    if (r < 0) r += d.n_bins;
    long long s0 = d.first_sample + r, end = (long long)d.first_sample + d.spp;
    fr->counts[fv][b] += s0 < end ? (end - 1 - s0) / d.n_bins + 1 : 0;
  }
}

}  // namespace

gr_status gr_render(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views, int32_t n_views,
                    const gr_render_opts* opts, gr_frame* frame, void* cuda_stream) {
  if (!frame) return fail(GR_E_INVALID, "gr_render: null frame");
  if (n_views != frame->n_views) return fail(GR_E_INVALID, "gr_render: view count differs from the frame's");
  std::vector<gr_frame*> frames(std::max(n_views, 1), frame);
  gr_status s = check_render_args("gr_render", scenes, n_scenes, views, n_views, opts, frames.data(), nullptr);
  if (s != GR_OK) return s;
  s = check_call_devices("gr_render", scenes, n_scenes, frames.data(), n_views);
  if (s != GR_OK) return s;
  std::vector<float*> as(n_views), ac(n_views);
  for (int v = 0; v < n_views; ++v) {
    as[v] = frame->acc + frame->offsets[v];
    ac[v] = frame->acc + frame->acc_floats + frame->offsets[v];
  }
  std::string err;
  s = gr::render_impl(scenes, n_scenes, views, n_views, *opts, frame, as, ac, (cudaStream_t)cuda_stream, err);
  if (s != GR_OK) return fail(s, "gr_render: " + err);
  for (int v = 0; v < n_views; ++v) add_counts(frame, v, views[v]);
  return GR_OK;
}

gr_status gr_render_multi(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views, int32_t n_views,
                          const gr_render_opts* opts, gr_frame* const* frames, const int32_t* frame_view,
                          void* cuda_stream) {
  if (!frame_view) return fail(GR_E_INVALID, "gr_render_multi: null frame_view");
  gr_status s = check_render_args("gr_render_multi", scenes, n_scenes, views, n_views, opts, frames, frame_view);
  if (s != GR_OK) return s;
  s = check_call_devices("gr_render_multi", scenes, n_scenes, frames, n_views);
  if (s != GR_OK) return s;
  std::vector<float*> as(n_views), ac(n_views);
  for (int v = 0; v < n_views; ++v) {
    gr_frame* fr = frames[v];
    as[v] = fr->acc + fr->offsets[frame_view[v]];
    ac[v] = fr->acc + fr->acc_floats + fr->offsets[frame_view[v]];
  }
  std::string err;
  s = gr::render_impl(scenes, n_scenes, views, n_views, *opts, frames[0], as, ac, (cudaStream_t)cuda_stream, err);
  if (s != GR_OK) return fail(s, "gr_render_multi: " + err);
  for (int v = 0; v < n_views; ++v) add_counts(frames[v], frame_view[v], views[v]);
  return GR_OK;
}

gr_status gr_render_scratch_bytes(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views,
                                  int32_t n_views, const gr_render_opts* opts, size_t* bytes_out) {
  if (!bytes_out || !views || n_views <= 0) return fail(GR_E_INVALID, "gr_render_scratch_bytes: null or empty argument");
  // the views' shapes are checked as a frame over them would check them
  std::vector<gr_view_shape> shapes;
  gr_frame probe;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = views[v];
    if (d.width <= 0 || d.height <= 0 || d.n_bins <= 0 || d.n_bins > 4096 || (d.n_stokes != 1 && d.n_stokes != 4))
      return fail(GR_E_INVALID, "gr_render_scratch_bytes: bad view shape " + std::to_string(v));
    probe.shapes.push_back(gr_view_shape{d.width, d.height, d.n_bins, d.n_stokes});
    probe.offsets.push_back(0);
  }
  probe.n_views = n_views;
  std::vector<gr_frame*> frames(n_views, &probe);
  gr_status s = check_render_args("gr_render_scratch_bytes", scenes, n_scenes, views, n_views, opts, frames.data(),
                                  nullptr);
  if (s != GR_OK) return s;
  std::vector<float*> none;
  std::string err;
  size_t bytes = 0;
  s = gr::render_impl(scenes, n_scenes, views, n_views, *opts, nullptr, none, none, nullptr, err, &bytes);
  if (s != GR_OK) return fail(s, "gr_render_scratch_bytes: " + err);
  *bytes_out = bytes;
  return GR_OK;
}

gr_status gr_readback(gr_frame* f, int32_t view, float* dst, size_t dst_bytes, int32_t dst_is_device, void* cuda_stream) {
  if (!f || !dst) return fail(GR_E_INVALID, "gr_readback: null argument");
  if (view < 0 || view >= f->n_views) return fail(GR_E_INVALID, "gr_readback: view out of range");
  const gr_view_shape& s = f->shapes[view];
  const size_t n = (size_t)s.W * s.H * s.nb * s.ns;
  if (dst_bytes < n * sizeof(float)) return fail(GR_E_INVALID, "gr_readback: destination too small");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  std::vector<float> inv(s.nb);
  for (int b = 0; b < s.nb; ++b) inv[b] = f->counts[view][b] > 0 ? 1.0f / (float)f->counts[view][b] : 0.0f;
  float* inv_d = nullptr;
  float* tmp = nullptr;
  cudaError_t e = cudaMallocAsync(&inv_d, sizeof(float) * s.nb, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(inv_d, inv.data(), sizeof(float) * s.nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !dst_is_device) e = cudaMallocAsync(&tmp, n * sizeof(float), st);
  if (e == cudaSuccess) e = gr::readback_impl(f, view, dst_is_device ? dst : tmp, inv_d, st);
  if (e == cudaSuccess && !dst_is_device) e = cudaMemcpyAsync(dst, tmp, n * sizeof(float), cudaMemcpyDeviceToHost, st);
  if (inv_d) cudaFreeAsync(inv_d, st);
  if (tmp) cudaFreeAsync(tmp, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // inv[] is pageable host memory; host dst must be complete
  if (e != cudaSuccess) return cuda_fail(e, "gr_readback");
  return GR_OK;
}

gr_status gr_frame_stats(gr_frame* f, void* cuda_stream, gr_stats* out) {
  if (!f || !out) return fail(GR_E_INVALID, "gr_frame_stats: null argument");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  gr::Counters c;
  cudaError_t e = cudaMemcpyAsync(&c, f->ctr, sizeof c, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "gr_frame_stats");
  out->samples = (int64_t)c.samples;
  out->segments = (int64_t)c.segments;
  out->shadow_rays = (int64_t)c.shadow;
  out->refine64_hits = (int64_t)c.ref_hit;
  out->refine64_lobes = (int64_t)c.ref_lobe;
  out->iterations = (int64_t)c.iters;
  out->kernel_launches = f->launches;
  out->node_visits = (int64_t)c.node_visits;
  out->tri_tests = (int64_t)c.tri_tests;
  for (int k = 0; k < 4; ++k) {
    out->kernel_ms[k] = f->kernel_ms[k];
    out->kernel_count[k] = f->kernel_launches[k];
  }
  return GR_OK;
}

gr_status gr_render_static(gr_scene* const* scenes, int32_t n_scenes, const gr_view_desc* views, int32_t n_views,
                           const gr_render_opts* opts, float* accum, void* cuda_stream) {
  if (!scenes || !views || !opts || !accum || n_views <= 0 || n_scenes <= 0)
    return fail(GR_E_INVALID, "gr_render_static: null or empty argument");
  if (opts->use_graph || opts->profile)
    return fail(GR_E_INVALID, "gr_render_static: use_graph and profile are not available without allocation");
  if (opts->flags & (GR_FLAG_HERO | GR_FLAG_ANISO))
    return fail(GR_E_INVALID,
                "gr_render_static: hero-wavelength MIS and anisotropic footprints are not available without allocation");
  for (int i = 0; i < n_scenes; ++i)
    if (!scenes[i]) return fail(GR_E_INVALID, "gr_render_static: null scene " + std::to_string(i));
  if (opts->table_dtype < GR_TABLE_F32 || opts->table_dtype > GR_TABLE_BF16)
    return fail(GR_E_INVALID, "gr_render_static: bad table dtype");
  if (opts->pool_size < 0 || opts->pool_size > gr::kMaxPool || opts->block < 0 ||
      (opts->block && (opts->block % 32 || opts->block > 256)))
    return fail(GR_E_INVALID, "gr_render_static: bad pool size (0 to 2^30 - 256) or block (a multiple of 32, <= 256)");
  if (opts->regen_threshold_pct < 0 || opts->regen_threshold_pct > 100)
    return fail(GR_E_INVALID, "gr_render_static: regen_threshold_pct out of [0, 100]");
  const int ns = views[0].n_stokes;
  for (int v = 0; v < n_views; ++v) {
    const gr_view_desc& d = views[v];
    if (d.width <= 0 || d.height <= 0 || d.n_bins <= 0 || d.n_bins > 4096 || (d.n_stokes != 1 && d.n_stokes != 4) ||
        (long long)d.width * d.height * d.n_bins >= (1LL << 31))
      return fail(GR_E_INVALID, "gr_render_static: bad view shape " + std::to_string(v));
    if (d.n_stokes != ns) return fail(GR_E_INVALID, "gr_render_static: all views of one call need the same n_stokes");
    if (d.scene_index < 0 || d.scene_index >= n_scenes)
      return fail(GR_E_INVALID, "gr_render_static: scene index out of range in view " + std::to_string(v));
    if (d.spp < 0 || d.first_sample < 0 || (long long)d.first_sample + d.spp >= (1LL << 31) ||
        (long long)d.spp / d.n_bins + 1 >= 65536)
      return fail(GR_E_INVALID, "gr_render_static: bad sample range in view " + std::to_string(v));
    if (d.max_depth < 0 || d.max_depth > 250) return fail(GR_E_INVALID, "gr_render_static: max_depth out of [0, 250]");
    if (!(d.lambda_min_um > 0.0f) || d.lambda_max_um < d.lambda_min_um || !(d.p_pix_um > 0.0f) || !(d.f_beta > 0.0f))
      return fail(GR_E_INVALID, "gr_render_static: bad spectral range or pixel footprint in view " + std::to_string(v));
    if (!(d.vfov_deg > 0.0f && d.vfov_deg < 180.0f) && !d.ortho)
      return fail(GR_E_INVALID, "gr_render_static: bad field of view in view " + std::to_string(v));
  }
  const int dev = current_device();
  if (dev < 0) return fail(GR_E_CUDA, "gr_render_static: no current CUDA device");
  gr_status s = check_scene_devices("gr_render_static", scenes, n_scenes, dev);
  if (s != GR_OK) return s;
  s = check_device_buffer("gr_render_static", accum, dev);
  if (s != GR_OK) return s;
  std::string err;
  s = gr::render_static_impl(scenes, n_scenes, views, n_views, *opts, accum, (cudaStream_t)cuda_stream, err);
  if (s != GR_OK) return fail(s, "gr_render_static: " + err);
  return GR_OK;
}

gr_status gr_debug_rng(uint32_t seed, uint32_t view_index, uint32_t pixel, uint32_t sample, int32_t segment,
                       int32_t call, int32_t n, uint32_t* out_u32, void* cuda_stream) {
  if (!out_u32 || n <= 0 || segment < 0 || segment > 0x0fffffff || call < 0 || call > 15)
    return fail(GR_E_INVALID, "gr_debug_rng: bad arguments");
  cudaError_t e = gr::debug_rng_impl(seed, view_index, pixel, sample, segment, call, n, out_u32,
                                     (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_debug_rng");
  return GR_OK;
}

gr_status gr_debug_order_table(float height_um, double lambda_um, int32_t jmax, int32_t table_dtype, float* out,
                               void* cuda_stream) {
  if (!out || jmax < 0 || jmax > 4096 || !(lambda_um > 0.0) || !(height_um >= 0.0f) ||
      (table_dtype != GR_TABLE_F32 && table_dtype != GR_TABLE_F16 && table_dtype != GR_TABLE_BF16))
    return fail(GR_E_INVALID, "gr_debug_order_table: bad arguments");
  cudaError_t e = gr::debug_table_impl(height_um, lambda_um, jmax, table_dtype, out, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_debug_order_table");
  return GR_OK;
}

gr_status gr_debug_footprint(int32_t n, const float* in, float* out, void* cuda_stream) {
  if (!in || !out || n <= 0) return fail(GR_E_INVALID, "gr_debug_footprint: bad arguments");
  cudaError_t e = gr::debug_footprint_impl(n, in, out, (cudaStream_t)cuda_stream);
  if (e != cudaSuccess) return cuda_fail(e, "gr_debug_footprint");
  return GR_OK;
}

gr_status gr_aperture_backward_2d(int32_t n_det, const double* x0, int32_t n_ap, const double* x_ap,
                                  const double* w_ap, double beta, double z, double k, double reach, double dtheta,
                                  double rho_cut, double* out, float* kernel_ms, void* cuda_stream) {
  if (!x0 || !x_ap || !w_ap || !out || n_det <= 0 || n_ap <= 0 || n_ap > 16384 || !(beta > 0.0) || !(z > 0.0) ||
      !(k > 0.0) || !(reach > 0.0) || !(dtheta > 0.0) || !(rho_cut > 0.0))
    return fail(GR_E_INVALID, "gr_aperture_backward_2d: bad arguments");
  // bound the direction grid: an element spans at most 2 atan(reach / z), in
  // at most 2^26 directions
  const double span = 2.0 * std::atan(reach / z);
  if (span / dtheta > (double)(1 << 26)) return fail(GR_E_INVALID, "gr_aperture_backward_2d: direction grid too fine");
  cudaError_t e = gr::aperture_backward_impl(n_det, x0, n_ap, x_ap, w_ap, beta, z, k, reach, dtheta, rho_cut, out,
                                             (cudaStream_t)cuda_stream, kernel_ms);
  if (e != cudaSuccess) return cuda_fail(e, "gr_aperture_backward_2d");
  return GR_OK;
}

gr_status gr_aperture_backward_3d(int32_t n_det, const double* x0, int32_t n_ap, const double* x_ap,
                                  const double* w_ap, double beta, double z, double k, double reach, double dt,
                                  double rho_cut, double* out, float* kernel_ms, void* cuda_stream) {
  if (!x0 || !x_ap || !w_ap || !out || n_det <= 0 || n_ap <= 0 || n_ap > 12288 || !(beta > 0.0) || !(z > 0.0) ||
      !(k > 0.0) || !(reach > 0.0) || !(dt > 0.0) || !(rho_cut > 0.0))
    return fail(GR_E_INVALID, "gr_aperture_backward_3d: bad arguments");
  // bound the direction grid: at most 2^13 directions per axis
  if (2.0 * reach / (z * dt) > (double)(1 << 13))
    return fail(GR_E_INVALID, "gr_aperture_backward_3d: direction grid too fine");
  cudaError_t e = gr::aperture_backward_3d_impl(n_det, x0, n_ap, x_ap, w_ap, beta, z, k, reach, dt, rho_cut, out,
                                                (cudaStream_t)cuda_stream, kernel_ms);
  if (e != cudaSuccess) return cuda_fail(e, "gr_aperture_backward_3d");
  return GR_OK;
}

}  // extern "C"
