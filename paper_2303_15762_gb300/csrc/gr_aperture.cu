// Footprint-resolved generalized rays through an aperture (the paper's
// double-slit validation, Sec. 5.1-5.2, in a 2D world, and its extension to a
// plane aperture in a 3D world below): a detector element is
// a coherent state of width beta at the screen (Eq. wdf_coherent_states); each
// of its directions theta is a generalized ray propagated back to the aperture
// plane in closed form (Eq. K_free_space_propagation over the oblique length
// z / cos(theta)), truncated to the ball of radius rho_cut beta' (Sec. 6), and
// overlapped with the sampled aperture field; the element's intensity is
// int dkappa / (2 pi) |<U_ap, psi_kappa>|^2 with kappa = k sin(theta).
//
// One block per detector element; its threads stride over the direction grid.
// Per-direction quantities are formed in FP64, the aperture sum in FP32 (the
// field samples are staged in shared memory), and the block's partial sums
// are reduced in a fixed order, so the result does not depend on scheduling.
#include <cuda_runtime.h>

#include <cmath>

#include "gr_build.h"

namespace gr {

namespace {

constexpr int kApertureThreads = 256;

// 2 pi split as hi + lo with hi the nearest float (Cody & Waite's additive
// range reduction): x - n (2 pi) is formed as (x - n hi) - n lo with one
// rounding per step, accurate to a few 1e-7 rad for |x| up to ~1e4.
constexpr float kTwoPiHi = 6.28318548202514648f;
constexpr float kTwoPiLo = -1.7484555314695172e-7f;
constexpr float kInvTwoPi = 0.159154943091895336f;

#ifndef GR_APERTURE_FAST_TRIG
#define GR_APERTURE_FAST_TRIG 1
#endif

// (cos x, sin x) for the overlap phases: reduced to [-pi, pi], then the
// hardware approximation (absolute error ~1e-6 there), below the ~6e-5 rad to
// which the FP32 phase itself is known.
__device__ __forceinline__ void phase_cis(float x, float* s, float* c) {
#if GR_APERTURE_FAST_TRIG
  const float n = rintf(x * kInvTwoPi);
  const float r = fmaf(-n, kTwoPiLo, fmaf(-n, kTwoPiHi, x));
  __sincosf(r, s, c);
#else
  sincosf(x, s, c);
#endif
}

__global__ void __launch_bounds__(kApertureThreads) k_aperture_backward(int n_det, const double* __restrict__ x0s,
                                                                        int n_ap, const float2* __restrict__ ap,
                                                                        double beta, double z, double k, double reach,
                                                                        double dtheta, double rho_cut,
                                                                        double* __restrict__ out) {
  extern __shared__ float2 s_ap[];  // (x, w) of every aperture sample
  __shared__ double s_red[kApertureThreads];
  for (int i = threadIdx.x; i < n_ap; i += blockDim.x) s_ap[i] = ap[i];
  __syncthreads();
  const double pi = 3.14159265358979323846;
  for (int det = blockIdx.x; det < n_det; det += gridDim.x) {
    const double x0 = x0s[det];
    const double th_lo = atan((x0 - reach) / z), th_hi = atan((x0 + reach) / z);
    const long long n_th = (long long)ceil((th_hi - th_lo) / dtheta);
    const double beta2 = beta * beta;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n_th; i += blockDim.x) {
      const double th = th_lo + (double)i * dtheta;
      const double c = cos(th), sn = sin(th);
      const double zb = (z / c) / k;                 // oblique path length over |k|
      const double b2 = beta2 + zb * zb / beta2;     // Eq. K_free_space_propagation from rho = 0
      const double rho = zb / beta2;
      const double xc = x0 - z * (sn / c);           // where the ray meets the aperture plane
      const float kap = (float)(k * sn), cf = (float)c, xcf = (float)xc;
      const float inv2b2 = (float)(0.5 / b2), rhof = (float)rho;
      const float cut = (float)(rho_cut * sqrt(b2));
      float re = 0.0f, im = 0.0f;
      for (int a = 0; a < n_ap; ++a) {
        const float2 q = s_ap[a];
        const float dx = q.x - xcf;
        const float u = dx * cf;
        if (fabsf(u) > cut) continue;
        const float u2 = u * u * inv2b2;
#if GR_APERTURE_FAST_TRIG
        const float g = q.y * __expf(-u2);
#else
        const float g = q.y * expf(-u2);
#endif
        float s, co;
        phase_cis(kap * dx - rhof * u2, &s, &co);
        re += g * co;
        im += g * s;
      }
      // |A|^2 with the state's normalisation (pi b'^2)^(-1/2) cos(theta), times dkappa
      const double amp2 = c / sqrt(pi * b2);
      acc += ((double)re * re + (double)im * im) * amp2 * (k * c * dtheta);
    }
    s_red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) s_red[threadIdx.x] += s_red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[det] = s_red[0] / (2.0 * pi);
    __syncthreads();
  }
}

// The same computation for a plane aperture in a 3D world: a detector element
// at (x0, y0) on the screen, directions on the tangent-plane grid t = (s_x,
// s_y) / s_z (landing points x_c = x0 - z t, one grid step apart), each a
// generalized ray propagated back over z / s_z in closed form, its footprint
// projected obliquely onto the aperture plane (|P d|^2 = |d|^2 - s_z^2 (t.d)^2)
// and truncated at rho_cut beta'; the element's intensity is
// sum_t |A|^2 s_z / (pi beta'^2) k^2 s_z^4 dt^2 / (2 pi)^2.  Aperture samples
// are (x, y, weight, 0) in shared memory.
__global__ void __launch_bounds__(kApertureThreads) k_aperture_backward_3d(int n_det, const double2* __restrict__ x0s,
                                                                           int n_ap, const float4* __restrict__ ap,
                                                                           double beta, double z, double k,
                                                                           double reach, double dt, double rho_cut,
                                                                           double* __restrict__ out) {
  extern __shared__ float4 s_ap4[];
  __shared__ double s_red[kApertureThreads];
  for (int i = threadIdx.x; i < n_ap; i += blockDim.x) s_ap4[i] = ap[i];
  __syncthreads();
  const double pi = 3.14159265358979323846;
  const long long n_t = (long long)ceil(2.0 * reach / (z * dt));
  const long long n_dir = n_t * n_t;
  const double beta2 = beta * beta;
  for (int det = blockIdx.x; det < n_det; det += gridDim.x) {
    const double2 x0 = x0s[det];
    const double tx0 = (x0.x - reach) / z, ty0 = (x0.y - reach) / z;
    double acc = 0.0;
    for (long long i = threadIdx.x; i < n_dir; i += blockDim.x) {
      const long long ix = i / n_t, iy = i - ix * n_t;
      const double tx = tx0 + (double)ix * dt, ty = ty0 + (double)iy * dt;
      const double sz = 1.0 / sqrt(1.0 + tx * tx + ty * ty);
      const double zb = (z / sz) / k;                // oblique path length over |k|
      const double b2 = beta2 + zb * zb / beta2;     // Eq. K_free_space_propagation from rho = 0
      const double rho = zb / beta2;
      const float cx = (float)(x0.x - z * tx), cy = (float)(x0.y - z * ty);
      const float kx = (float)(k * sz * tx), ky = (float)(k * sz * ty);
      const float txf = (float)tx, tyf = (float)ty, sz2 = (float)(sz * sz);
      const float inv2b2 = (float)(0.5 / b2), rhof = (float)rho;
      const float cut2 = (float)(rho_cut * rho_cut * b2);
      float re = 0.0f, im = 0.0f;
      for (int a = 0; a < n_ap; ++a) {
        const float4 q = s_ap4[a];
        const float dx = q.x - cx, dy = q.y - cy;
        const float td = txf * dx + tyf * dy;
        const float p2 = fmaf(dx, dx, dy * dy) - sz2 * td * td;
        if (p2 > cut2) continue;
        const float u2 = p2 * inv2b2;
#if GR_APERTURE_FAST_TRIG
        const float g = q.z * __expf(-u2);
#else
        const float g = q.z * expf(-u2);
#endif
        float s, co;
        phase_cis(fmaf(kx, dx, ky * dy) - rhof * u2, &s, &co);
        re += g * co;
        im += g * s;
      }
      const double amp2 = sz / (pi * b2);
      acc += ((double)re * re + (double)im * im) * amp2 * (k * k * sz * sz * sz * sz * dt * dt);
    }
    s_red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) s_red[threadIdx.x] += s_red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) out[det] = s_red[0] / (4.0 * pi * pi);
    __syncthreads();
  }
}

}  // namespace

cudaError_t aperture_backward_3d_impl(int n_det, const double* x0_host, int n_ap, const double* xa_host,
                                      const double* wa_host, double beta, double z, double k, double reach,
                                      double dt, double rho_cut, double* out_host, cudaStream_t st, float* ms) {
  double2* d_x0 = nullptr;
  double* d_out = nullptr;
  float4* d_ap = nullptr;
  float4* h_ap = nullptr;
  cudaError_t e = cudaMallocHost(&h_ap, sizeof(float4) * (size_t)n_ap);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < n_ap; ++i)
    h_ap[i] = make_float4((float)xa_host[2 * i], (float)xa_host[2 * i + 1], (float)wa_host[i], 0.0f);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMallocAsync(&d_x0, sizeof(double2) * (size_t)n_det, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_out, sizeof(double) * (size_t)n_det, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_ap, sizeof(float4) * (size_t)n_ap, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_x0, x0_host, sizeof(double2) * (size_t)n_det, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ap, h_ap, sizeof(float4) * (size_t)n_ap, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int grid = 1;
  const size_t smem = sizeof(float4) * (size_t)n_ap;
  if (e == cudaSuccess) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = n_det < sms * 8 ? n_det : sms * 8;
    if (smem > 48 * 1024)
      e = cudaFuncSetAttribute(k_aperture_backward_3d, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e == cudaSuccess) {
    cudaEventRecord(e0, st);
    k_aperture_backward_3d<<<grid, kApertureThreads, smem, st>>>(n_det, d_x0, n_ap, d_ap, beta, z, k, reach, dt,
                                                                 rho_cut, d_out);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, d_out, sizeof(double) * (size_t)n_det, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_x0) cudaFreeAsync(d_x0, st);
  if (d_out) cudaFreeAsync(d_out, st);
  if (d_ap) cudaFreeAsync(d_ap, st);
  cudaStreamSynchronize(st);
  cudaFreeHost(h_ap);
  return e;
}

cudaError_t aperture_backward_impl(int n_det, const double* x0_host, int n_ap, const double* xa_host,
                                   const double* wa_host, double beta, double z, double k, double reach,
                                   double dtheta, double rho_cut, double* out_host, cudaStream_t st, float* ms) {
  double* d_x0 = nullptr;
  double* d_out = nullptr;
  float2* d_ap = nullptr;
  float2* h_ap = nullptr;
  cudaError_t e = cudaMallocHost(&h_ap, sizeof(float2) * (size_t)n_ap);
  if (e != cudaSuccess) return e;
  for (int i = 0; i < n_ap; ++i) h_ap[i] = make_float2((float)xa_host[i], (float)wa_host[i]);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMallocAsync(&d_x0, sizeof(double) * (size_t)n_det, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_out, sizeof(double) * (size_t)n_det, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_ap, sizeof(float2) * (size_t)n_ap, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_x0, x0_host, sizeof(double) * (size_t)n_det, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_ap, h_ap, sizeof(float2) * (size_t)n_ap, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  int grid = 1;
  if (e == cudaSuccess) {
    int dev = 0, sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    grid = n_det < sms * 8 ? n_det : sms * 8;
    const size_t smem = sizeof(float2) * (size_t)n_ap;
    if (smem > 48 * 1024)
      e = cudaFuncSetAttribute(k_aperture_backward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  }
  if (e == cudaSuccess) {
    cudaEventRecord(e0, st);
    k_aperture_backward<<<grid, kApertureThreads, sizeof(float2) * (size_t)n_ap, st>>>(
        n_det, d_x0, n_ap, d_ap, beta, z, k, reach, dtheta, rho_cut, d_out);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out_host, d_out, sizeof(double) * (size_t)n_det, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && ms) e = cudaEventElapsedTime(ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d_x0) cudaFreeAsync(d_x0, st);
  if (d_out) cudaFreeAsync(d_out, st);
  if (d_ap) cudaFreeAsync(d_ap, st);
  cudaStreamSynchronize(st);
  cudaFreeHost(h_ap);
  return e;
}

}  // namespace gr
