// Internal interface between the warm-start network's host code (dtt_net.cu) and its
// kernels (k_net.cu).
#pragma once
#include <cuda_bf16.h>

#include "dtt_internal.cuh"

namespace dtt {
namespace net {

constexpr int CF_RELU = 1;   // ReLU on the conv output
constexpr int CF_SKIP = 2;   // then add a skip tensor (the ReLU output is also stored in r)
constexpr int CF_F32 = 4;    // FP32 output, no activation
constexpr int NET_CIN = 16;  // input feature channels (13 used)
constexpr int NET_COUT = 16; // output channels of the last layer (3 used)

struct ConvArgs {
  int cin, cout, flags;
  int nx, ny, nz;
  const __nv_bfloat16* x;     // [V][cin] layer input
  const __nv_bfloat16* wt;    // [27][cout][cin]
  const __nv_bfloat16* wd;    // [27][cin][cout]
  const float* bias;          // [cout]
  __nv_bfloat16* y;           // [V][cout] output (BF16 flags)
  float* yf;                  // [V][cout] output (CF_F32)
  const __nv_bfloat16* skip;  // [V][cout] (CF_SKIP)
  __nv_bfloat16* r;           // [V][cout] ReLU output before the skip (CF_SKIP)
  // backward
  const __nv_bfloat16* dz;    // [V][cout] gradient at the conv output (pre-activation)
  float* dx;                  // [V][cin] gradient at the input (may be null)
  float* dw;                  // [27][cout][cin] accumulated
  float* db;                  // [cout] accumulated
};

// A box of the node grid: origin o and extent n (the whole grid: o = 0, n = nn).
struct Window {
  int o[3];
  int n[3];
};

struct FeatArgs {
  GridDev g;
  Window w;             // nodes whose features are written, x indexed inside the window
  const uint8_t* phase;
  const float* enorm;   // E / E_max per phase
  const uint8_t* cmask;
  float eps6[6];        // eps* xx yy zz yz xz xy, times 1000
  float* x;             // [Vw][16]
};

// Increment mode (one load increment of a sphere indentation, Algorithm 2): features
// built from the previous increments' fields, targets of the displacement correction and
// of the contact pressure, and the guess written back (layout in include/dtt_net.h).
struct IncArgs {
  GridDev g;
  Window w;              // the network's window (features, targets and outputs inside it)
  const double* u64;     // u~ of increment k-1 (FP64 grid) ...
  const float* uhi;      // ... or its float-float pair (mixed grid)
  const float* ulo;
  const double* u2;      // u~ of increment k-2 (device, [3][V]; null: zero)
  double s_sec;          // secant factor of the increment (d^(3/2) steps)
  double dd;             // depth increment d_k - d_(k-1) (> 0)
  int nface;
  const long long* node; // surface nodes
  const double* fn_prev; // normal reactions of increment k-1 at the surface nodes
  const uint8_t* fn_act; // if set: fn_prev counts only where fn_act[q] != 0 (the grid's own contact set)
  double center[3];      // sphere centre of increment k
  double radius;
  double eps[3][3];
  float* fmax;           // device scalar: max over the surface of -fn_prev (set by launch_inc_fmax)
  float* x;              // [Vw][16] features (base channels already written)
};
// normal reaction of increment k-1 at surface node q (zero off its contact set)
__device__ inline double inc_fn(const IncArgs& a, int q) {
  return (a.fn_act && !a.fn_act[q]) ? 0.0 : a.fn_prev[q];
}
__host__ __device__ inline long long win_volume(const Window& w) { return (long long)w.n[0] * w.n[1] * w.n[2]; }
int launch_inc_fmax(const IncArgs& a, cudaStream_t s);
int launch_inc_features(const IncArgs& a, cudaStream_t s);
// targets t[V][4] (displacement correction, pressure) and the pressure mask m[V]
int launch_inc_targets(const IncArgs& a, const double* u_target, const double* fn_target, float* t, float* m,
                       cudaStream_t s);
int launch_inc_loss(const float* y, const float* t, const float* m, long long V, int CY, float wp, float* gy,
                    double* loss, cudaStream_t s);
// guess u = u~_(k-1) + dd (x[4..6] + y[0..2]) into u[3][V]; active[q] = fn_prev[q] < 0 or
// y[node q][3] > thr
int launch_inc_guess(const IncArgs& a, const float* y, int CY, float thr, double* u, uint8_t* active,
                     cudaStream_t s);

int launch_conv_fwd(const ConvArgs& a, cudaStream_t s);
int launch_conv_bwd(const ConvArgs& a, cudaStream_t s);
int launch_relu_bwd(const float* G, const __nv_bfloat16* R, long long n, __nv_bfloat16* dZ, cudaStream_t s);
int launch_pool_fwd(const __nv_bfloat16* in, int nx, int ny, int nz, int C, __nv_bfloat16* out, cudaStream_t s);
int launch_pool_bwd_add(const float* gc, int nx, int ny, int nz, int C, float* gf, cudaStream_t s);
int launch_up_fwd(const __nv_bfloat16* coarse, int nx, int ny, int nz, int C, __nv_bfloat16* fine, cudaStream_t s);
int launch_up_bwd(const float* gf, int nx, int ny, int nz, int C, float* gc, cudaStream_t s);
int launch_add(float* a, const float* b, long long n, cudaStream_t s);
int launch_f2bf(const float* a, long long n, __nv_bfloat16* b, cudaStream_t s);
int launch_loss(const float* y, const float* t, int nx, int ny, int nz, int CY, float s2, float* gy, double* loss,
                cudaStream_t s);
int launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s,
                float gscale = 1.f);
int launch_relayout(const float* W, int cin, int cout, __nv_bfloat16* Wt, __nv_bfloat16* Wd, cudaStream_t s);
int launch_features(const FeatArgs& a, cudaStream_t s);
int launch_out_to_u(const float* y, long long V, int CY, double scale, double* u, cudaStream_t s);

}  // namespace net
}  // namespace dtt
