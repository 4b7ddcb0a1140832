// Fused z pass (forward DTT along z, Green multiply, inverse DTT along z) as two dense
// contractions on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Along z the transform of one component is a dense product with a fixed matrix (Section
// 3.2.2: the DCT/DST of Table 3 written out as the matrix of its trigonometric sums, F for
// the forward and B for the inverse, each restricted to the active nodes and spectral
// positions of the component's type).  For a tile of 128 z-pencils (one per tensor-memory
// lane) the pass computes
//   D1 = X F^T              (pencil m, spectral k)   -- GEMM 1
//   Z  = D1 / a_c(q)        (Green multiply, 0 on null modes)
//   D2 = Z B^T              (pencil m, node j)       -- GEMM 2
// with X[m][j] the pencil values.  Both products run in kind::tf32 with each operand split
// into a TF32 high part and an FP32 remainder (x = hi + lo, hi = x with its low 13 mantissa
// bits cleared): hi.hi + hi.lo + lo.hi keeps about 21 bits of each product, the accuracy
// of the FP32 FFT pass it replaces, and the accumulators are FP32 in tensor memory.
//
// Data movement: the pencil values are gathered by all threads with coalesced loads (32
// consecutive pencils per warp and z plane), split and written to shared memory in the
// canonical no-swizzle K-major layout (core matrices of 8 rows x 16 bytes); the constant
// matrices are stored in global memory already in that layout, chunk by chunk, and each
// chunk arrives by one bulk asynchronous copy completing on an mbarrier.  Chunks of 32
// along K are double-buffered, so the tensor core works on one chunk while the threads
// fill the next.  The epilogue of GEMM 1 reads D1 from tensor memory, applies the Green
// symbol (the same FP32 expression as the FFT pass) and produces GEMM 2's operand chunks
// in the same pipeline; the epilogue of GEMM 2 writes the node values back with coalesced
// stores.  Every wait is bounded: on a timeout the CTA records an error word, skips the
// rest of its work, waits (bounded) for its outstanding tensor-core work, frees its tensor
// memory and returns.
#include <cstdint>
#include <cstring>
#include <vector>

#include "dtt_internal.cuh"

namespace dtt {

namespace {

constexpr int TZ_M = 128;         // pencils per CTA (tensor-memory lanes)
constexpr int TZ_KC = 32;         // K chunk (floats)
constexpr int TZ_THREADS = 256;   // 8 warps: two per tensor-memory lane quarter
constexpr uint32_t TZ_TMEM_COLS = 512;

// byte offset of element (row r, k) inside one operand chunk (rows x 32 floats), canonical
// K-major layout without swizzle: core matrix (8 rows x 4 floats, 128 contiguous bytes)
// at (r / 8, k / 4); core matrices along K 128 bytes apart (leading byte offset), groups
// of 8 rows 1024 bytes apart (stride byte offset)
__host__ __device__ __forceinline__ uint32_t tz_off(int r, int k) {
  return (uint32_t)((r >> 3) * 1024 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start address, leading byte offset 128 (K direction),
// stride byte offset 1024 (8-row groups), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tz_desc(uint32_t saddr) {
  return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(1024 >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::tf32: D FP32, A and B TF32, both K-major, M = 128, N
__host__ __device__ constexpr uint32_t tz_idesc(int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(TZ_M >> 4) << 24);
}

__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Bounded wait for the completion of the phase with parity `parity`; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done = 0;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;   // about one second at 2 GHz
  }
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
// 16 consecutive 32-bit columns of this thread's lane
__device__ __forceinline__ void tc_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}

template <typename T>
__device__ __forceinline__ T tz_tetra_S(T sa, T cb, T sb, T cA, T sc) {
  const T d = (sa + sb < (T)1) ? (sb - sa) : (cA - cb);
  return sa * cb + sc * d;
}

}  // namespace

// 16 floats of one row into an operand chunk: hi part to `hi`, remainder to `lo`
__device__ __forceinline__ void tz_put16(unsigned char* hi, unsigned char* lo, int r, int k0, const float* v) {
#pragma unroll
  for (int q = 0; q < 16; q += 4) {
    float4 h, l;
    h.x = tf32_hi(v[q]);
    h.y = tf32_hi(v[q + 1]);
    h.z = tf32_hi(v[q + 2]);
    h.w = tf32_hi(v[q + 3]);
    l.x = v[q] - h.x;
    l.y = v[q + 1] - h.y;
    l.z = v[q + 2] - h.z;
    l.w = v[q + 3] - h.w;
    const uint32_t o = tz_off(r, k0 + q);
    *(float4*)(hi + o) = h;
    *(float4*)(lo + o) = l;
  }
}

// NC = P / 32 operand chunks (compile time: the pencil values of GEMM 1 are gathered into
// registers in one batch of 16 NC loads per thread before the first chunk is written, so
// that the whole tile's loads are in flight together)
template <int NC>
__global__ void __launch_bounds__(TZ_THREADS, 1)
k_tz_green(const float* __restrict__ in, float* __restrict__ out, TzParams p, GreenTables gt, float l0, float m2,
           float ih2, int scheme, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  extern __shared__ __align__(1024) unsigned char tz_smem[];
  __shared__ __align__(8) uint64_t bfull[2], mdone[2], drain;
  __shared__ uint32_t tmem_slot;
  __shared__ int s_err;
  const int comp = p.comp0 + blockIdx.y;
  const TzComp& cp = p.c[comp];
  constexpr int P = NC * TZ_KC;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int m = tid & (TZ_M - 1);        // pencil row = tensor-memory lane
  const int half = tid >> 7;             // which 16 of a 32-wide chunk this thread handles
  const long long pen = (long long)blockIdx.x * TZ_M + m;
  const bool valid = pen < p.npencil;
  const long long base = (long long)comp * p.NN + (valid ? pen : 0);
  const long long stride = p.stride;

  // shared memory: A stages [2][hi, lo][128 x 32], B stages [2][hi, lo][P x 32], z tables
  unsigned char* As = tz_smem;
  const uint32_t a_bytes = TZ_M * TZ_KC * 4;          // 16 KB per part
  unsigned char* Bs = As + 2 * 2 * a_bytes;
  const uint32_t b_bytes = (uint32_t)P * TZ_KC * 4;   // per part
  float* zs = (float*)(Bs + 2 * 2 * b_bytes);
  float* zc = zs + P;

  if (tid == 0) {
    mbar_init(&bfull[0], 1);
    mbar_init(&bfull[1], 1);
    mbar_init(&mdone[0], 1);
    mbar_init(&mdone[1], 1);
    mbar_init(&drain, 1);
    s_err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_slot)),
                 "r"(TZ_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  for (int k = tid; k < P; k += TZ_THREADS) {
    const bool in_range = k < cp.nk;
    zs[k] = in_range ? gt.sf[comp][2][cp.k0 + k] : 0.f;
    zc[k] = in_range ? gt.cpf[comp][2][cp.k0 + k] : 1.f;
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t lane_base = (uint32_t)((warp & 3) * 32) << 16;
  const uint32_t d1 = tmem, d2 = tmem + (uint32_t)P;
  const uint32_t idesc = tz_idesc(P);

  // per-pencil symbol factors (x and y already transformed)
  float sx = 0.f, cx = 1.f, sy = 0.f, cy = 1.f;
  if (valid) {
    const int ix = (int)(pen % p.nnx), iy = (int)(pen / p.nnx);
    sx = gt.sf[comp][0][ix];
    cx = gt.cpf[comp][0][ix];
    sy = gt.sf[comp][1][iy];
    cy = gt.cpf[comp][1][iy];
  }
  const float thr = gt.null_thr_f[comp];

  // One pipelined contraction: chunk g (global count over both GEMMs) uses stage g & 1.
  // produce(cidx, hi, lo) writes A chunk cidx; the matrix chunk comes by bulk copy.
  auto run_gemm = [&](int g0, const unsigned char* mat, uint32_t dcol, auto produce) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const int g = g0 + c, s = g & 1;
      if (g >= 2 && !s_err) {
        if (!mbar_wait(&mdone[s], (uint32_t)(((g - 2) >> 1) & 1))) s_err = 1;
      }
      __syncthreads();
      if (s_err) return;
      unsigned char* ahi = As + (2 * s) * a_bytes;
      unsigned char* alo = ahi + a_bytes;
      unsigned char* bhi = Bs + (2 * s) * b_bytes;
      if (tid == 0) {
        mbar_expect_tx(&bfull[s], 2 * b_bytes);
        bulk_g2s(bhi, mat + (size_t)c * 2 * b_bytes, 2 * b_bytes, &bfull[s]);
      }
      produce(c, ahi, alo);
      fence_async_smem();
      tc_fence_before();
      __syncthreads();
      if (tid == 0) {
        if (!mbar_wait(&bfull[s], (uint32_t)((g >> 1) & 1))) {
          s_err = 1;
        } else {
          tc_fence_after();
          const uint32_t a0 = smem_u32(ahi), l0a = smem_u32(alo);
          const uint32_t b0 = smem_u32(bhi), l0b = smem_u32(bhi + b_bytes);
#pragma unroll
          for (int kk = 0; kk < TZ_KC / 8; ++kk) {
            const uint32_t o = kk * 256;   // two core matrices along K per instruction
            tc_mma(dcol, tz_desc(a0 + o), tz_desc(b0 + o), idesc, (c | kk) != 0);
            tc_mma(dcol, tz_desc(a0 + o), tz_desc(l0b + o), idesc, 1);
            tc_mma(dcol, tz_desc(l0a + o), tz_desc(b0 + o), idesc, 1);
          }
          tc_commit(&mdone[s]);
        }
      }
    }
  };
  // every thread waits for the last chunk of a contraction (its commit covers all earlier
  // tensor-core work) before reading the accumulators
  auto wait_last = [&](int g_last) {
    if (!s_err && !mbar_wait(&mdone[g_last & 1], (uint32_t)((g_last >> 1) & 1))) s_err = 1;
    tc_fence_after();
    __syncthreads();
  };

  // ---- GEMM 1: D1 = X F^T
  float xv[NC][16];
#pragma unroll
  for (int c = 0; c < NC; ++c)
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int k = c * TZ_KC + half * 16 + q;
      xv[c][q] = (valid && k < cp.nj) ? __ldg(in + base + (long long)(cp.j0 + k) * stride) : 0.f;
    }
  run_gemm(0, (const unsigned char*)cp.fwd, d1, [&](int c, unsigned char* hi, unsigned char* lo) {
    tz_put16(hi, lo, m, half * 16, xv[c]);
  });
  wait_last(NC - 1);

  // ---- Green multiply (epilogue 1) feeding GEMM 2: D2 = Z B^T
  run_gemm(NC, (const unsigned char*)cp.inv, d2, [&](int c, unsigned char* hi, unsigned char* lo) {
    float v[16];
    const int kb = c * TZ_KC + half * 16;
    tc_ld16(d1 + lane_base + (uint32_t)kb, v);
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int k = kb + q;
      const float sz = zs[k], cz = zc[k];
      float Sx, Sy, Sz;
      if (scheme == SCHEME_TETRA2) {
        Sx = tz_tetra_S<float>(sx, cy, sy, cx, sz);
        Sy = tz_tetra_S<float>(sy, cz, sz, cy, sx);
        Sz = tz_tetra_S<float>(sz, cx, sx, cz, sy);
      } else {
        Sx = sx * cy * cz;
        Sy = sy * cx * cz;
        Sz = sz * cx * cy;
      }
      const float Sc = comp == 0 ? Sx : (comp == 1 ? Sy : Sz);
      const float a = (l0 * Sc + m2 * (Sx + Sy + Sz)) * ih2;
      v[q] = (k >= cp.nk || a <= thr) ? 0.f : v[q] / a;
    }
    tz_put16(hi, lo, m, half * 16, v);
  });
  wait_last(2 * NC - 1);

  // ---- epilogue 2: node values of the active rows, zeros on the others
  if (!s_err) {
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      float v[16];
      const int nb = c * TZ_KC + half * 16;
      tc_ld16(d2 + lane_base + (uint32_t)nb, v);
      if (valid) {
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          const int n = nb + q;
          if (n < cp.nj) out[base + (long long)(cp.j0 + n) * stride] = v[q];
        }
      }
    }
    if (valid)
      for (int j = half; j < p.nnz; j += 2)
        if (j < cp.j0 || j >= cp.j0 + cp.nj) out[base + (long long)j * stride] = 0.f;
  } else {
    // a wait timed out: record it, and let outstanding tensor-core work drain (bounded)
    // before the tensor memory is released
    if (tid == 0) {
      atomicOr(p.err, 1u);
      tc_commit(&drain);   // arrives once every MMA this thread issued has completed
      mbar_wait(&drain, 0);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TZ_TMEM_COLS)
                 : "memory");
  }
}

template <int NC>
static int tz_launch(dim3 grid, size_t sm, const float* in, float* out, const TzParams& p, const GreenTables& gt,
                     float l0, float m2, float ih2, int scheme, const Ctrl* ctrl, cudaStream_t s) {
  static size_t done = 0;   // per instance: the largest dynamic shared memory granted so far
  if (sm > done) {
    cudaError_t e = cudaFuncSetAttribute(k_tz_green<NC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return (int)e;
    done = sm;
  }
  k_tz_green<NC><<<grid, TZ_THREADS, sm, s>>>(in, out, p, gt, l0, m2, ih2, scheme, ctrl);
  return (int)cudaGetLastError();
}

size_t tz_smem_bytes(int P) {
  return (size_t)2 * 2 * TZ_M * TZ_KC * 4 + (size_t)2 * 2 * P * TZ_KC * 4 + (size_t)2 * P * 4;
}

int launch_tz_green(const float* in, float* out, const TzParams& p, const GreenTables& gt, double lam0, double mu0,
                    int scheme, double h, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  int P = 0;
  for (int c = p.comp0; c < p.comp0 + ncomp; ++c) P = p.c[c].P > P ? p.c[c].P : P;
  for (int c = p.comp0; c < p.comp0 + ncomp; ++c)
    if (p.c[c].P != P) return (int)cudaErrorInvalidValue;   // one shared-memory plan per launch
  if (P < TZ_KC || P > 256 || P % TZ_KC) return (int)cudaErrorInvalidValue;
  const size_t sm = tz_smem_bytes(P);
  const float l0 = (float)lam0, m2 = (float)(2.0 * mu0), ih2 = (float)(4.0 / (h * h));
  dim3 grid((unsigned)((p.npencil + TZ_M - 1) / TZ_M), (unsigned)ncomp);
  switch (P / TZ_KC) {
    case 1: return tz_launch<1>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 2: return tz_launch<2>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 3: return tz_launch<3>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 4: return tz_launch<4>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 5: return tz_launch<5>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 6: return tz_launch<6>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 7: return tz_launch<7>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    case 8: return tz_launch<8>(grid, sm, in, out, p, gt, l0, m2, ih2, scheme, ctrl, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

// Host side: the operand chunks of one component's matrices in the layout above.  For
// chunk q (K range [32 q, 32 q + 32)) the hi part (P x 32) is followed by the lo part.
void tz_pack_matrix(const double* M, int nn, int r0, int nr, int c0, int ncol, int P, std::vector<float>& outv) {
  const int NC = P / TZ_KC;
  const size_t part = (size_t)P * TZ_KC;   // floats
  outv.assign((size_t)NC * 2 * part, 0.f);
  for (int q = 0; q < NC; ++q) {
    float* hi = outv.data() + (size_t)q * 2 * part;
    float* lo = hi + part;
    for (int r = 0; r < P; ++r)
      for (int kl = 0; kl < TZ_KC; ++kl) {
        const int k = q * TZ_KC + kl;
        const double v = (r < nr && k < ncol) ? M[(size_t)(r0 + r) * nn + (c0 + k)] : 0.0;
        const float f = (float)v;
        uint32_t bits;
        std::memcpy(&bits, &f, 4);
        bits &= 0xFFFFE000u;
        float h;
        std::memcpy(&h, &bits, 4);
        const size_t o = tz_off(r, kl) / 4;
        hi[o] = h;
        lo[o] = f - h;
      }
  }
}

}  // namespace dtt
