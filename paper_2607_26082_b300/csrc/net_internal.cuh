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

struct FeatArgs {
  GridDev g;
  const uint8_t* phase;
  const float* enorm;   // E / E_max per phase
  const uint8_t* cmask;
  float eps6[6];        // eps* xx yy zz yz xz xy, times 1000
  float* x;             // [V][16]
};

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
int launch_adam(float* p, const float* g, float* m, float* v, long long n, float lr, int step, cudaStream_t s);
int launch_relayout(const float* W, int cin, int cout, __nv_bfloat16* Wt, __nv_bfloat16* Wd, cudaStream_t s);
int launch_features(const FeatArgs& a, cudaStream_t s);
int launch_out_to_u(const float* y, long long V, int CY, double scale, double* u, cudaStream_t s);

}  // namespace net
}  // namespace dtt
