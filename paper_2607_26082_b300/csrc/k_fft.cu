// Fast per-axis DTTs: two real pencils of the same component and axis packed into one
// complex sequence, one shared-memory Stockham FFT (radices 4, 2, 3), and type-specific
// pre/post-processing.  O(n log n) per pencil instead of the O(n^2) dense contraction.
//
// With z = a + i b (a, b two real pencils, node values x_j) and L the FFT length:
//   DCT1 (L = 2n): even extension y_j = z_j, y_{2n-j} = z_j;  X_a = Re Y / 2, X_b = Im Y / 2.
//   DST1 (L = 2n): odd extension, y_0 = y_n = 0;             X_a = -Im Y / 2, X_b = Re Y / 2.
//   DCT3 (L = 2n): odd extension about n, y_n = 0, times e^{-i pi j / 2n}; Re / Im as DCT1.
//   DST3 (L = 2n): even extension about n, y_0 = 0, times e^{-i pi j / 2n}; as DST1.
//   Hartley (L = n, periodic axis): H_a = (u + u' - v + v') / 2, H_b = (u - u' + v + v') / 2
//     with Y_k = u + i v, Y_{(n-k) mod n} = u' + i v'.
// (Y = DFT of the extended sequence; e.g. the DFT of the even extension is 2 X for DCT1, and
// the modulated quarter-wave extensions give 2 X exactly, so the pair separates without
// further work.)  The inverses of DCT1, DST1 and the Hartley transform are the forward
// formulas times 2/n (1/n); the inverses of DCT3 / DST3 take the length-2n unnormalised
// inverse DFT of X extended as X_{2n-1-k} = +-X_k and read x_j from e^{+i pi j / 2n} Z_j / n.
// These follow from the trigonometric sums of the transforms (Section 3.2.2, Tables 2-3);
// the 4n-extended DFT of Eq. 7 is the same idea with the redundant half removed.
#include <cstdlib>
#include <type_traits>

#include "dtt_internal.cuh"

namespace dtt {

// Aligned to its full size, so that a complex value is one 64-bit (FP32) or 128-bit (FP64)
// access: every array of them starts at a cudaMalloc base or a 16-byte-aligned shared offset.
template <typename T> struct __align__(2 * sizeof(T)) Cx { T x, y; };

template <typename T>
__device__ __forceinline__ Cx<T> cmul(Cx<T> a, Cx<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}

// R-point DFT in registers, sign s = -1 (forward) or +1 (inverse, unnormalised).
template <typename T>
__device__ __forceinline__ void dft2(Cx<T>* v) {
  Cx<T> a = v[0], b = v[1];
  v[0] = {a.x + b.x, a.y + b.y};
  v[1] = {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ void dft4(Cx<T>* v, int s) {
  Cx<T> a = {v[0].x + v[2].x, v[0].y + v[2].y}, b = {v[0].x - v[2].x, v[0].y - v[2].y};
  Cx<T> c = {v[1].x + v[3].x, v[1].y + v[3].y}, d = {v[1].x - v[3].x, v[1].y - v[3].y};
  // w d with w = s i:  s (-d.y + i d.x)
  Cx<T> wd = {(T)(-s) * d.y, (T)s * d.x};
  v[0] = {a.x + c.x, a.y + c.y};
  v[2] = {a.x - c.x, a.y - c.y};
  v[1] = {b.x + wd.x, b.y + wd.y};
  v[3] = {b.x - wd.x, b.y - wd.y};
}
template <typename T>
__device__ __forceinline__ void dft3(Cx<T>* v, int s) {
  const T c = (T)-0.5, sn = (T)s * (T)0.86602540378443864676;
  Cx<T> t1 = {v[1].x + v[2].x, v[1].y + v[2].y}, t2 = {v[1].x - v[2].x, v[1].y - v[2].y};
  Cx<T> m = {v[0].x + c * t1.x, v[0].y + c * t1.y};
  // i sn t2 = (-sn t2.y, sn t2.x)
  v[0] = {v[0].x + t1.x, v[0].y + t1.y};
  v[1] = {m.x - sn * t2.y, m.y + sn * t2.x};
  v[2] = {m.x + sn * t2.y, m.y - sn * t2.x};
}

// One Stockham stage of radix R for all PB sequences of the CTA (registers only).  lgLR /
// lgNs are log2 of L/R and Ns when L is a power of two (shift and mask index math), else -1.
template <typename T, int R>
__device__ __forceinline__ void stockham_stage(const Cx<T>* __restrict__ S, Cx<T>* __restrict__ D, int L, int Ns,
                                               int PBL, const Cx<T>* __restrict__ tw, int sgn, int tid, int nthr,
                                               int lgLR, int lgNs) {
  const int LR = L / R;
  const int twstep = L / (Ns * R);
  for (int idx = tid; idx < PBL / R; idx += nthr) {
    int q, jb, k;
    if (lgLR >= 0) {
      q = idx >> lgLR;
      jb = idx & (LR - 1);
      k = jb & (Ns - 1);
    } else {
      q = idx / LR;
      jb = idx - q * LR;
      k = jb % Ns;
    }
    const Cx<T>* Sq = S + q * L;
    Cx<T>* Dq = D + q * L;
    Cx<T> v[R];
    #pragma unroll
    for (int r = 0; r < R; ++r) v[r] = Sq[jb + r * LR];
    #pragma unroll
    for (int r = 1; r < R; ++r) {
      Cx<T> w = tw[k * r * twstep];   // k r twstep < L
      if (sgn > 0) w.y = -w.y;
      v[r] = cmul(v[r], w);
    }
    if constexpr (R == 4) dft4(v, sgn);
    else if constexpr (R == 2) dft2(v);
    else dft3(v, sgn);
    const int o = (jb - k) * R + k;
    #pragma unroll
    for (int r = 0; r < R; ++r) Dq[o + r * Ns] = v[r];
  }
}

template <typename T>
__device__ __forceinline__ T tetra_S(T sa, T cb, T sb, T cA, T sc) {
  const T d = (sa + sb < (T)1) ? (sb - sa) : (cA - cb);
  return sa * cb + sc * d;
}

// ---- building blocks of one CTA's work on PB pencil pairs --------------------------------

// Extended (and, for quarter-wave forward types, modulated) complex sequences of the CTA
// in A, from values get(pb, j) of pencil pb (0..2PB-1) at axis position j (0..nn-1).
// rowwise: a warp reads one pencil at consecutive j (pencils contiguous in memory, x axis);
// otherwise consecutive threads take consecutive pencils at the same j (y and z axes, whose
// neighbouring pencils are neighbours in memory).
template <typename T, int PB, typename Get>
__device__ __forceinline__ void fill_sequences(Cx<T>* A, int L, int n, int nn, int type, int inverse, int npen,
                                               const Cx<T>* ph, Get get, int tid, int nthr, bool rowwise) {
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  for (int q = tid; q < PB; q += nthr) {
    Cx<T>* S = A + q * L;
    if (!inverse || !quarter) {
      if (type == T_DST1) { S[0] = {(T)0, (T)0}; S[n] = {(T)0, (T)0}; }
      else if (type == T_DCT3) S[n] = {(T)0, (T)0};
      else if (type == T_DST3) S[0] = {(T)0, (T)0};
    }
  }
  if (npen < 2 * PB)
    for (int q = tid; q < PB * L; q += nthr) A[q] = {(T)0, (T)0};
  __syncthreads();
  auto place = [&](int pb, int j, T v) {
    Cx<T>* S = A + (pb >> 1) * L;
    const bool im = pb & 1;
    auto put = [&](int pos, T val) {
      if (im) S[pos].y = val; else S[pos].x = val;
    };
    if (!inverse || !quarter) {
      switch (type) {
        case T_DCT1:
          put(j, v);
          if (j >= 1 && j <= n - 1) put(2 * n - j, v);
          break;
        case T_DST1:
          if (j >= 1 && j <= n - 1) { put(j, v); put(2 * n - j, -v); }
          break;
        case T_DCT3:
          if (j <= n - 1) { put(j, v); if (j >= 1) put(2 * n - j, -v); }
          break;
        case T_DST3:
          if (j >= 1) { put(j, v); if (j <= n - 1) put(2 * n - j, v); }
          break;
        default:
          put(j, v);
          break;
      }
    } else if (j < n) {
      put(j, v);
      put(2 * n - 1 - j, type == T_DCT3 ? v : -v);
    }
  };
  if (rowwise) {
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    for (int pb = warp; pb < npen; pb += nw)
      for (int j = lane; j < nn; j += 32) place(pb, j, get(pb, j));
  } else {
    for (int idx = tid; idx < 2 * PB * nn; idx += nthr) {
      const int pb = idx % (2 * PB), j = idx / (2 * PB);
      if (pb >= npen) continue;
      place(pb, j, get(pb, j));
    }
  }
  __syncthreads();
  if (quarter && !inverse) {
    for (int j = tid; j < L; j += nthr) {
      const Cx<T> w = ph[j];
      #pragma unroll
      for (int q = 0; q < PB; ++q) A[q * L + j] = cmul(A[q * L + j], w);
    }
    __syncthreads();
  }
}

// Stockham FFT of the PB sequences; returns the buffer holding the result.
template <typename T, int PB>
__device__ __forceinline__ Cx<T>* fft_sequences(Cx<T>* s0, Cx<T>* s1, const FftParams& p, const Cx<T>* tw, int sgn,
                                                int tid, int nthr) {
  const bool pow2 = (p.L & (p.L - 1)) == 0;
  const int lgL = pow2 ? __ffs(p.L) - 1 : -1;
  int Ns = 1, lgNs = 0;
  for (int st = 0; st < p.nst; ++st) {
    const int R = p.radix[st];
    const int lgR = R == 4 ? 2 : (R == 2 ? 1 : -1);
    const int lgLR = pow2 ? lgL - lgR : -1;
    const int lns = pow2 ? lgNs : -1;
    if (R == 4) stockham_stage<T, 4>(s0, s1, p.L, Ns, PB * p.L, tw, sgn, tid, nthr, lgLR, lns);
    else if (R == 2) stockham_stage<T, 2>(s0, s1, p.L, Ns, PB * p.L, tw, sgn, tid, nthr, lgLR, lns);
    else stockham_stage<T, 3>(s0, s1, p.L, Ns, PB * p.L, tw, sgn, tid, nthr, -1, -1);
    __syncthreads();
    Cx<T>* t = s0;
    s0 = s1;
    s1 = t;
    Ns *= R;
    if (lgR > 0) lgNs += lgR;
  }
  return s0;
}

// Transform value of pencil pb at spectral / node position k from the FFT result Y.
template <typename T>
__device__ __forceinline__ T post_value(const Cx<T>* Yall, int L, int n, int type, int inverse, T sc, const Cx<T>* ph,
                                        int pb, int k, T inv_n) {
  const Cx<T>* Y = Yall + (pb >> 1) * L;
  const bool im = pb & 1;
  const T half = (T)0.5;
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  if (!inverse || !quarter) {
    T val = (T)0;
    switch (type) {
      case T_DCT1:
        val = im ? half * Y[k].y : half * Y[k].x;
        break;
      case T_DST1:
        if (k >= 1 && k <= n - 1) val = im ? half * Y[k].x : -half * Y[k].y;
        break;
      case T_DCT3:
        if (k <= n - 1) val = im ? half * Y[k].y : half * Y[k].x;
        break;
      case T_DST3:
        if (k <= n - 1) val = im ? half * Y[k].x : -half * Y[k].y;
        break;
      default: {
        const Cx<T> a = Y[k], b = Y[k == 0 ? 0 : n - k];
        val = im ? half * (a.x - b.x + a.y + b.y) : half * (a.x + b.x - a.y + b.y);
        break;
      }
    }
    return val * sc;
  }
  const Cx<T> w = {ph[k].x, -ph[k].y};
  const Cx<T> e = cmul(Y[k], w);
  if (type == T_DCT3) return (k <= n - 1) ? (im ? e.y : e.x) * inv_n : (T)0;
  return (k >= 1) ? (im ? -e.x : e.y) * inv_n : (T)0;
}

template <typename T, int PB>
__device__ __forceinline__ void pencil_bases(long long* sbase, const FftParams& p, long long pen0, int tid) {
  if (tid < 2 * PB) {
    const long long pen = pen0 + tid;
    long long b = 0;
    if (pen < p.npencil) {
      if (p.axis == 0) b = pen * p.nnx;
      else if (p.axis == 1) b = (pen / p.nnx) * (long long)p.nnx * p.nny + (pen % p.nnx);
      else b = pen;
    }
    sbase[tid] = b;
  }
}

template <typename T>
__device__ __forceinline__ void add_to_u(long long e, T val, const FftParams& p) {
  if constexpr (sizeof(T) == 8) {
    p.u64[e] += (double)val;
  } else {
    float h = p.uhi[e], l = p.ulo[e];
    ff_add(h, l, (float)val);
    p.uhi[e] = h;
    p.ulo[e] = l;
  }
  if (p.step) ((T*)p.step)[e] = val;
}

// Shared-memory layout of one CTA: two buffers of PB sequences of length L, then the L
// twiddles, then (z pass) per-position symbol tables.
template <typename T, int PB>
__host__ __device__ constexpr size_t fft_smem_base(int L) {
  return (size_t)(2 * PB + 1) * (size_t)L * sizeof(Cx<T>);
}

// One axis pass: forward or inverse DTT of every pencil along p.axis.  With p.incr (inverse
// x pass), the result is added to u~ and written as the step instead of to `out`.
template <typename T, int PB>
__global__ void __launch_bounds__(256)
k_fft_axis(const T* __restrict__ in, T* __restrict__ out, FftParams p, const Ctrl* ctrl, void* const* in_ring) {
  if (ctrl && ctrl->done) return;
  if (in_ring) in = (const T*)in_ring[ctrl->i_local % 4];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long sbase[2 * PB];
  Cx<T>* bufA = (Cx<T>*)smem_raw;
  Cx<T>* bufB = bufA + PB * p.L;
  Cx<T>* tws = bufB + PB * p.L;
  const Cx<T>* tw = (const Cx<T>*)p.tw;
  const Cx<T>* ph = (const Cx<T>*)p.ph;
  const int comp = p.comp0 + blockIdx.y;
  const int type = p.type[comp];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const long long pen0 = (long long)blockIdx.x * (2 * PB);
  const T* src = in + (long long)comp * p.NN;
  const long long coff = (long long)comp * p.NN;
  const long long stride = p.axis == 0 ? 1 : (p.axis == 1 ? (long long)p.nnx : (long long)p.nnx * p.nny);
  const int npen = (int)min((long long)(2 * PB), p.npencil - pen0);
  const bool rowwise = p.axis == 0;
  pencil_bases<T, PB>(sbase, p, pen0, tid);
  for (int q = tid; q < p.L; q += nthr) tws[q] = tw[q];
  __syncthreads();
  fill_sequences<T, PB>(bufA, p.L, p.n, p.nn, type, p.inverse, npen, ph,
                        [&](int pb, int j) { return src[sbase[pb] + j * stride]; }, tid, nthr, rowwise);
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  const int sgn = (p.inverse && quarter) ? 1 : -1;
  Cx<T>* Y = fft_sequences<T, PB>(bufA, bufB, p, tws, sgn, tid, nthr);
  const T sc = sizeof(T) == 4 ? (T)p.fscale : (T)p.scale;
  const T inv_n = sizeof(T) == 4 ? (T)p.finv_n : (T)p.inv_n;
  auto emit = [&](int pb, int k) {
    const T v = post_value<T>(Y, p.L, p.n, type, p.inverse, sc, ph, pb, k, inv_n);
    const long long e = coff + sbase[pb] + k * stride;
    if (p.incr) add_to_u<T>(e, v, p);
    else out[e] = v;
  };
  if (rowwise) {
    const int warp = tid >> 5, lane = tid & 31, nw = nthr >> 5;
    for (int pb = warp; pb < npen; pb += nw)
      for (int k = lane; k < p.nn; k += 32) emit(pb, k);
  } else {
    for (int idx = tid; idx < 2 * PB * p.nn; idx += nthr) {
      const int pb = idx % (2 * PB), k = idx / (2 * PB);
      if (pb >= npen) continue;
      emit(pb, k);
    }
  }
}

// Fused z pass: forward DTT along z, Green multiply (Eq. 4 adapted to the Paux reference,
// Section 3.2.3), inverse DTT along z, for pencils whose x and y spectra are already taken.
// The symbol factors sin^2(q/2), cos^2(q/2) of the z positions are staged in shared memory
// once per CTA, those of the CTA's pencils (x and y positions) once per pencil.
template <typename T, int PB>
__global__ void __launch_bounds__(256)
k_fft_z_green(const T* __restrict__ in, T* __restrict__ out, FftParams p, GreenTables gt, T l0, T m2, T ih2,
              int scheme, T zscale, const Ctrl* ctrl) {
  if (ctrl && ctrl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long sbase[2 * PB];
  __shared__ T pxy[2 * PB][4];   // per pencil: s_x, c'_x, s_y, c'_y
  Cx<T>* bufA = (Cx<T>*)smem_raw;
  Cx<T>* bufB = bufA + PB * p.L;
  Cx<T>* tws = bufB + PB * p.L;
  T* zs = (T*)(tws + p.L);        // s_z[k], k < nn
  T* zc = zs + p.nn;              // c'_z[k]
  const Cx<T>* tw = (const Cx<T>*)p.tw;
  const Cx<T>* ph = (const Cx<T>*)p.ph;
  const int comp = p.comp0 + blockIdx.y;
  const int type = p.type[comp];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const long long pen0 = (long long)blockIdx.x * (2 * PB);
  const long long coff = (long long)comp * p.NN;
  const long long stride = (long long)p.nnx * p.nny;
  const int npen = (int)min((long long)(2 * PB), p.npencil - pen0);
  const int nn = p.nn;
  pencil_bases<T, PB>(sbase, p, pen0, tid);
  if (tid < 2 * PB) {
    const long long pen = pen0 + tid;
    const int ix = pen < p.npencil ? (int)(pen % p.nnx) : 0, iy = pen < p.npencil ? (int)(pen / p.nnx) : 0;
    pxy[tid][0] = gt_s<T>(gt, comp, 0, ix);
    pxy[tid][1] = gt_c<T>(gt, comp, 0, ix);
    pxy[tid][2] = gt_s<T>(gt, comp, 1, iy);
    pxy[tid][3] = gt_c<T>(gt, comp, 1, iy);
  }
  for (int q = tid; q < p.L; q += nthr) tws[q] = tw[q];
  for (int q = tid; q < nn; q += nthr) {
    zs[q] = gt_s<T>(gt, comp, 2, q);
    zc[q] = gt_c<T>(gt, comp, 2, q);
  }
  __syncthreads();
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  const T inv_n = sizeof(T) == 4 ? (T)p.finv_n : (T)p.inv_n;
  // forward along z
  fill_sequences<T, PB>(bufA, p.L, p.n, nn, type, 0, npen, ph,
                        [&](int pb, int j) { return in[coff + sbase[pb] + j * stride]; }, tid, nthr, false);
  Cx<T>* Y = fft_sequences<T, PB>(bufA, bufB, p, tws, -1, tid, nthr);
  Cx<T>* I = (Y == bufA) ? bufB : bufA;
  T* spec = (T*)I;   // 2 PB x nn real spectra (fits in one complex buffer)
  const T thr = sizeof(T) == 4 ? (T)gt.null_thr_f[comp] : (T)gt.null_thr[comp];
  for (int idx = tid; idx < 2 * PB * nn; idx += nthr) {
    const int pb = idx % (2 * PB), k = idx / (2 * PB);
    T v = (T)0;
    if (pb < npen) {
      v = post_value<T>(Y, p.L, p.n, type, 0, (T)1, ph, pb, k, inv_n);
      const T sx = pxy[pb][0], cx = pxy[pb][1], sy = pxy[pb][2], cy = pxy[pb][3];
      const T sz = zs[k], cz = zc[k];
      T Sx, Sy, Sz;
      if (scheme == SCHEME_TETRA2) {
        Sx = tetra_S<T>(sx, cy, sy, cx, sz);
        Sy = tetra_S<T>(sy, cz, sz, cy, sx);
        Sz = tetra_S<T>(sz, cx, sx, cz, sy);
      } else {
        Sx = sx * cy * cz;
        Sy = sy * cx * cz;
        Sz = sz * cx * cy;
      }
      const T Sc = comp == 0 ? Sx : (comp == 1 ? Sy : Sz);
      const T a = (l0 * Sc + m2 * (Sx + Sy + Sz)) * ih2;
      v = (a <= thr) ? (T)0 : v / a;
    }
    spec[pb * nn + k] = v;
  }
  __syncthreads();
  // inverse along z
  Cx<T>* X = Y;
  fill_sequences<T, PB>(X, p.L, p.n, nn, type, 1, npen, ph, [&](int pb, int j) { return spec[pb * nn + j]; }, tid,
                        nthr, false);
  Y = fft_sequences<T, PB>(X, I, p, tws, quarter ? 1 : -1, tid, nthr);
  for (int idx = tid; idx < 2 * PB * nn; idx += nthr) {
    const int pb = idx % (2 * PB), k = idx / (2 * PB);
    if (pb >= npen) continue;
    out[coff + sbase[pb] + k * stride] = post_value<T>(Y, p.L, p.n, type, 1, zscale, ph, pb, k, inv_n);
  }
}

// ==== register-radix route: L = 2^k (16..2048) or 3 * 2^k (48..1536), compile-time L =====
//
// L / 8 threads own one complex sequence.  The power-of-two factor of L goes through
// radix-8 passes (radix 4 or 2 for the rest), each loading 8 values per thread from shared
// memory, applying the Stockham twiddles and a DFT in registers, and writing back in place
// between two barriers; a factor 3 adds one last radix-3 pass, in which a thread takes 2 or
// 3 of the L / 3 butterflies.  The sequences live in shared memory as a real and an
// imaginary array; FastMap<L> places element i of sequence seq so that the warps' strided
// accesses (the Stockham writes, the column-wise fills and reads of several pencils at one
// position) spread over the 32 banks.  A CTA holds 2048 complex values on 256 threads
// (power of two) or 1536 on 192 threads (3 * 2^k): SEQ sequences, twice as many real pencils.

template <int L>
struct FastPlan {
  static constexpr bool POW2 = (L & (L - 1)) == 0;
  static constexpr int P2 = POW2 ? L : L / 3;             // power-of-two factor
  static constexpr int NT = L / 8;                        // threads per sequence
  static constexpr int SEQ = (POW2 ? 2048 : 1536) / L;    // sequences per CTA
  static constexpr int THREADS = NT * SEQ;                // 256 or 192
  static constexpr int MINB = POW2 ? 5 : 6;               // fused z pass: CTAs per SM
  static_assert(POW2 || (P2 & (P2 - 1)) == 0, "L must be 2^k or 3 * 2^k");
};

// Shared-memory word of element i of sequence seq in array arr (0 real, 1 imaginary):
//     seq * PADL + i + (i >> S) * A + (i >> T) * B,   PADL = L + (L >> S) * A + (L >> T) * B + EXTRA,
// the imaginary array SEQ * PADL + OFF words after the real one.  The padding constants
// are chosen per length from a simulation of every warp access of the fills, the Stockham
// passes and the reads (x and y axes); simulated wavefronts against the former one word
// per 32 (S = 5, A = 1) and the bound of one wavefront per warp instruction:
//     L      16     32     64    128    256    512   1024   2048
//     now  1992   1800   2306   3297   2258   2257   2773   2787
//     was 12160   4104   4036   4388   3352   3344   3852   3462
//     bound 1992  1604   1538   1985   1954   1938   2442   2438
template <int L>
struct FastMapParams {
  static constexpr int S = 5, A = 2, T = 7, B = 1, EXTRA = 0, OFF = 0;   // 256 and up
};
template <> struct FastMapParams<16> { static constexpr int S = 3, A = 1, T = 0, B = 0, EXTRA = 0, OFF = 1; };
template <> struct FastMapParams<32> { static constexpr int S = 3, A = 1, T = 0, B = 0, EXTRA = 0, OFF = 1; };
template <> struct FastMapParams<64> { static constexpr int S = 5, A = 3, T = 0, B = 0, EXTRA = 0, OFF = 1; };
template <> struct FastMapParams<128> { static constexpr int S = 5, A = 2, T = 0, B = 0, EXTRA = 1, OFF = 0; };
// 3 * 2^k (192 threads), simulated the same way; wavefronts against the power-of-two default:
//     L       48     96    192    384    768
//     now   1874   2162   2420   2783   2081
//     was   3060   2978   2785   2974   2214
template <> struct FastMapParams<48> { static constexpr int S = 5, A = 3, T = 0, B = 0, EXTRA = 19, OFF = 1; };
template <> struct FastMapParams<96> { static constexpr int S = 5, A = 3, T = 0, B = 0, EXTRA = 3, OFF = 1; };
template <> struct FastMapParams<192> { static constexpr int S = 5, A = 3, T = 0, B = 0, EXTRA = 0, OFF = 0; };
template <> struct FastMapParams<384> { static constexpr int S = 5, A = 3, T = 0, B = 0, EXTRA = 15, OFF = 0; };
template <> struct FastMapParams<768> { static constexpr int S = 5, A = 3, T = 0, B = 0, EXTRA = 0, OFF = 0; };

template <int L>
struct FastMap {
  using P = FastMapParams<L>;
  static constexpr int SEQ = FastPlan<L>::SEQ;
  static constexpr int PADL = L + (L >> P::S) * P::A + (P::T ? (L >> P::T) * P::B : 0) + P::EXTRA;
  static constexpr int ARR = SEQ * PADL + P::OFF;
  static constexpr int WORDS = (2 * ARR + 3) & ~3;   // both arrays, 16-byte multiple
  __device__ static __forceinline__ int at(int arr, int seq, int i) {
    return arr * ARR + seq * PADL + i + (i >> P::S) * P::A + (P::T ? (i >> P::T) * P::B : 0);
  }
};

// 8-point DFT with kernel e^{s 2 pi i j k / 8}, natural-order output (decimation in
// frequency; the bit-reversed result is reordered in registers).
template <typename T>
__device__ __forceinline__ void dft8(Cx<T>* v, int s) {
  const T h = (T)0.70710678118654752440;
  const T sf = (T)s;
  Cx<T> a[8];
  #pragma unroll
  for (int j = 0; j < 4; ++j) {
    a[j] = {v[j].x + v[j + 4].x, v[j].y + v[j + 4].y};
    a[j + 4] = {v[j].x - v[j + 4].x, v[j].y - v[j + 4].y};
  }
  // a[4 + j] *= w^j, w = e^{s 2 pi i / 8}
  {
    const Cx<T> b = a[5];
    a[5] = {h * (b.x - sf * b.y), h * (sf * b.x + b.y)};
    const Cx<T> c = a[6];
    a[6] = {-sf * c.y, sf * c.x};
    const Cx<T> d = a[7];
    a[7] = {h * (-d.x - sf * d.y), h * (sf * d.x - d.y)};
  }
  #pragma unroll
  for (int hb = 0; hb < 8; hb += 4) {
    #pragma unroll
    for (int j = 0; j < 2; ++j) {
      const Cx<T> x = a[hb + j], y = a[hb + j + 2];
      a[hb + j] = {x.x + y.x, x.y + y.y};
      const Cx<T> d = {x.x - y.x, x.y - y.y};
      a[hb + j + 2] = j ? Cx<T>{-sf * d.y, sf * d.x} : d;
    }
  }
  #pragma unroll
  for (int p = 0; p < 8; p += 2) {
    const Cx<T> x = a[p], y = a[p + 1];
    a[p] = {x.x + y.x, x.y + y.y};
    a[p + 1] = {x.x - y.x, x.y - y.y};
  }
  v[0] = a[0]; v[4] = a[1]; v[2] = a[2]; v[6] = a[3];
  v[1] = a[4]; v[5] = a[5]; v[3] = a[6]; v[7] = a[7];
}

// Radix of the register-radix pass at stride NS (0: past the last pass).
template <int L, int NS>
__host__ __device__ constexpr int fast_radix() {
  constexpr int P2 = FastPlan<L>::P2;
  return (NS * 8 <= P2) ? 8 : (NS * 4 == P2) ? 4 : (NS * 2 == P2) ? 2 : (NS == P2 && P2 != L) ? 3 : 0;
}

// Pass twiddles in shared memory, pass after pass, each as [k][r - 1] (k < NS, 1 <= r < R):
// entry w(k, r) = e^{-2 pi i k r / (NS R)} is copied from the length-L table at k r L / (NS R).
// The threads of a warp take consecutive k, so one r reads NS-strided words in the
// length-L table (bank conflicts) but a stride of R - 1 here.  The tables hold at most L
// entries in all.  OFF is the start of the pass at stride NS.
template <int L, int NS = 1>
__host__ __device__ constexpr int fast_tw_off() {
  if constexpr (NS == 1) {
    return 0;
  } else {
    // sum over the passes before stride NS: strides NS' > 1 with radix R'
    int off = 0;
    int ns = 1;
    while (ns < NS) {
      const int r = (ns * 8 <= FastPlan<L>::P2) ? 8 : (ns * 4 == FastPlan<L>::P2) ? 4 : (ns * 2 == FastPlan<L>::P2) ? 2 : 3;
      if (ns > 1) off += ns * (r - 1);
      ns *= r;
    }
    return off;
  }
}

template <typename T, int L, int NS = 1>
__device__ __forceinline__ void fast_tw_fill(Cx<T>* twp, const Cx<T>* __restrict__ tw, int tid, int nthr) {
  constexpr int R = fast_radix<L, NS>();
  if constexpr (R != 0) {
    if constexpr (NS > 1) {
      constexpr int TWS = L / (NS * R), CNT = NS * (R - 1), OFF = fast_tw_off<L, NS>();
      for (int q = tid; q < CNT; q += nthr) {
        const int k = q / (R - 1), r = q - k * (R - 1) + 1;
        twp[OFF + q] = tw[k * r * TWS];
      }
    }
    fast_tw_fill<T, L, NS * R>(twp, tw, tid, nthr);
  }
}

// One in-place Stockham pass of radix R (stride NS) over the CTA's sequences; thread t of
// sequence `seq` takes butterflies t, t + NT, ... (8 / R of them).  With `mod`, the inputs
// are first multiplied by mod[index] (quarter-wave modulation of the forward transforms).
// tw: the pass twiddle tables of fast_tw_fill.
template <typename T, int L, int R, int NS>
__device__ __forceinline__ void fast_pass(T* buf, const Cx<T>* __restrict__ tw, int sgn, int seq, int t,
                                          const Cx<T>* __restrict__ mod) {
  using M = FastMap<L>;
  constexpr int NT = FastPlan<L>::NT;
  constexpr int LR = L / R, PER = 8 / R, OFF = fast_tw_off<L, NS>();
  Cx<T> v[PER][R];
  #pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int jb = t + m * NT;
    const int k = jb & (NS - 1);
    #pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = jb + r * LR;
      v[m][r] = {buf[M::at(0, seq, idx)], buf[M::at(1, seq, idx)]};
      if (mod) v[m][r] = cmul(v[m][r], mod[idx]);
    }
    if (NS > 1) {
      #pragma unroll
      for (int r = 1; r < R; ++r) {
        Cx<T> w = tw[OFF + k * (R - 1) + (r - 1)];
        if (sgn > 0) w.y = -w.y;
        v[m][r] = cmul(v[m][r], w);
      }
    }
    if constexpr (R == 8) dft8(v[m], sgn);
    else if constexpr (R == 4) dft4(v[m], sgn);
    else dft2(v[m]);
  }
  __syncthreads();
  #pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int jb = t + m * NT;
    const int k = jb & (NS - 1);
    const int o = (jb - k) * R + k;
    #pragma unroll
    for (int r = 0; r < R; ++r) {
      const int idx = o + r * NS;
      buf[M::at(0, seq, idx)] = v[m][r].x;
      buf[M::at(1, seq, idx)] = v[m][r].y;
    }
  }
  __syncthreads();
}

// The last Stockham pass of L = 3 * NS: L / 3 radix-3 butterflies over the NT = L / 8
// threads of a sequence, thread t taking t, t + NT and (for t < L / 12) t + 2 NT.
template <typename T, int L, int NS>
__device__ __forceinline__ void fast_pass3(T* buf, const Cx<T>* __restrict__ tw, int sgn, int seq, int t) {
  using M = FastMap<L>;
  constexpr int NT = FastPlan<L>::NT;
  constexpr int LR = L / 3, PER = (LR + NT - 1) / NT, OFF = fast_tw_off<L, NS>();
  static_assert(NS * 3 == L && PER == 3, "radix-3 pass closes 3 * 2^k");
  Cx<T> v[PER][3];
  #pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int jb = t + m * NT;
    if (m < PER - 1 || jb < LR) {
      const int k = jb & (NS - 1);
      #pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int idx = jb + r * LR;
        v[m][r] = {buf[M::at(0, seq, idx)], buf[M::at(1, seq, idx)]};
      }
      #pragma unroll
      for (int r = 1; r < 3; ++r) {
        Cx<T> w = tw[OFF + k * 2 + (r - 1)];
        if (sgn > 0) w.y = -w.y;
        v[m][r] = cmul(v[m][r], w);
      }
      dft3(v[m], sgn);
    }
  }
  __syncthreads();
  #pragma unroll
  for (int m = 0; m < PER; ++m) {
    const int jb = t + m * NT;
    if (m < PER - 1 || jb < LR) {
      const int k = jb & (NS - 1);
      const int o = (jb - k) * 3 + k;
      #pragma unroll
      for (int r = 0; r < 3; ++r) {
        const int idx = o + r * NS;
        buf[M::at(0, seq, idx)] = v[m][r].x;
        buf[M::at(1, seq, idx)] = v[m][r].y;
      }
    }
  }
  __syncthreads();
}

// Whole FFT of length L: radix-8 passes over the power-of-two factor P2, one radix-4 or
// radix-2 pass for the rest of it, then the radix-3 pass when L = 3 P2.  Every stride NS is
// a power of two, so the butterfly's offset k within its group is jb & (NS - 1).
template <typename T, int L, int NS = 1>
__device__ __forceinline__ void fast_fft(T* buf, const Cx<T>* tw, int sgn, int seq, int t, const Cx<T>* mod) {
  constexpr int P2 = FastPlan<L>::P2;
  if constexpr (NS * 8 <= P2) {
    fast_pass<T, L, 8, NS>(buf, tw, sgn, seq, t, NS == 1 ? mod : nullptr);
    fast_fft<T, L, NS * 8>(buf, tw, sgn, seq, t, nullptr);
  } else if constexpr (NS * 4 == P2) {
    fast_pass<T, L, 4, NS>(buf, tw, sgn, seq, t, NS == 1 ? mod : nullptr);
    fast_fft<T, L, NS * 4>(buf, tw, sgn, seq, t, nullptr);
  } else if constexpr (NS * 2 == P2) {
    fast_pass<T, L, 2, NS>(buf, tw, sgn, seq, t, NS == 1 ? mod : nullptr);
    fast_fft<T, L, NS * 2>(buf, tw, sgn, seq, t, nullptr);
  } else if constexpr (NS == P2 && P2 != L) {
    fast_pass3<T, L, NS>(buf, tw, sgn, seq, t);
  }
}

// Runs f with the transform type as a compile-time constant: the CTA's type is uniform, so
// the per-value branches of the extension and the post-processing fold away.
template <typename F>
__device__ __forceinline__ void by_type(int type, F&& f) {
  switch (type) {
    case T_DCT1: f(std::integral_constant<int, T_DCT1>()); break;
    case T_DCT3: f(std::integral_constant<int, T_DCT3>()); break;
    case T_DST1: f(std::integral_constant<int, T_DST1>()); break;
    case T_DST3: f(std::integral_constant<int, T_DST3>()); break;
    default: f(std::integral_constant<int, T_DHT>()); break;
  }
}

// Value v of real pencil pb at axis position j into the extended sequence of its pair (the
// same extensions as fill_sequences), in the real / imaginary arrays of the buffer.
template <typename T, int L>
__device__ __forceinline__ void fast_place(T* buf, int pb, int j, T v, int n, int type, int inverse) {
  const int arr = pb & 1, seq = pb >> 1;
  auto S = [&](int i) -> T& { return buf[FastMap<L>::at(arr, seq, i)]; };
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  if (!inverse || !quarter) {
    switch (type) {
      case T_DCT1:
        S(j) = v;
        if (j >= 1 && j <= n - 1) S(2 * n - j) = v;
        break;
      case T_DST1:
        if (j >= 1 && j <= n - 1) { S(j) = v; S(2 * n - j) = -v; }
        break;
      case T_DCT3:
        if (j <= n - 1) { S(j) = v; if (j >= 1) S(2 * n - j) = -v; }
        break;
      case T_DST3:
        if (j >= 1) { S(j) = v; if (j <= n - 1) S(2 * n - j) = v; }
        break;
      default:
        S(j) = v;
        break;
    }
  } else if (j < n) {
    S(j) = v;
    S(2 * n - 1 - j) = type == T_DCT3 ? v : -v;
  }
}

// The positions of pencil pb's extended sequence that fast_place leaves unwritten, set to
// zero (instead of clearing the whole buffer before the fill): 0 and n for DST1, n for the
// forward DCT3 extension, 0 for the forward DST3 extension.  DCT1, the Hartley sequence and
// the inverse quarter-wave extensions write every position.
template <typename T, int L, int TY>
__device__ __forceinline__ void fast_holes(T* buf, int pb, int n, int inverse) {
  const int arr = pb & 1, seq = pb >> 1;
  if (TY == T_DST1) {
    buf[FastMap<L>::at(arr, seq, 0)] = (T)0;
    buf[FastMap<L>::at(arr, seq, n)] = (T)0;
  } else if (TY == T_DCT3 && !inverse) {
    buf[FastMap<L>::at(arr, seq, n)] = (T)0;
  } else if (TY == T_DST3 && !inverse) {
    buf[FastMap<L>::at(arr, seq, 0)] = (T)0;
  }
}

// Transform value of pencil pb at position k from the FFT result of its pair (post_value on
// the padded arrays).
template <typename T, int L>
__device__ __forceinline__ T fast_post(const T* buf, int pb, int k, int n, int type, int inverse, T sc,
                                       const Cx<T>* ph, T inv_n) {
  const int seq = pb >> 1;
  auto yr = [&](int i) { return buf[FastMap<L>::at(0, seq, i)]; };
  auto yi = [&](int i) { return buf[FastMap<L>::at(1, seq, i)]; };
  const bool imf = pb & 1;
  const T half = (T)0.5;
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  if (!inverse || !quarter) {
    T val = (T)0;
    switch (type) {
      case T_DCT1:
        val = half * (imf ? yi(k) : yr(k));
        break;
      case T_DST1:
        if (k >= 1 && k <= n - 1) val = imf ? half * yr(k) : -half * yi(k);
        break;
      case T_DCT3:
        if (k <= n - 1) val = half * (imf ? yi(k) : yr(k));
        break;
      case T_DST3:
        if (k <= n - 1) val = imf ? half * yr(k) : -half * yi(k);
        break;
      default: {
        const int kk = k == 0 ? 0 : n - k;
        const T ax = yr(k), ay = yi(k), bx = yr(kk), by = yi(kk);
        val = imf ? half * (ax - bx + ay + by) : half * (ax + bx - ay + by);
        break;
      }
    }
    return val * sc;
  }
  const Cx<T> w = {ph[k].x, -ph[k].y};
  const Cx<T> e = cmul(Cx<T>{yr(k), yi(k)}, w);
  if (type == T_DCT3) return (k <= n - 1) ? (imf ? e.y : e.x) * inv_n : (T)0;
  return (k >= 1) ? (imf ? -e.x : e.y) * inv_n : (T)0;
}

// Row pb and position j of element idx of a block of consecutive rows of nn values
// (idx < 2^23): a float estimate of the quotient, off by at most one, then corrected.
__device__ __forceinline__ void row_pos(int idx, int nn, float rnn, int& pb, int& j) {
  int q = __float2int_rz((float)idx * rnn);
  int r = idx - q * nn;
  if (r < 0) {
    --q;
    r += nn;
  } else if (r >= nn) {
    ++q;
    r -= nn;
  }
  pb = q;
  j = r;
}

template <typename T, int L>
__host__ __device__ constexpr size_t fast_smem(int extra_bytes) {
  return (size_t)FastMap<L>::WORDS * sizeof(T) + (size_t)L * sizeof(Cx<T>) +
         (size_t)extra_bytes;
}

// Axis pass on the register-radix route (same contract as k_fft_axis).
template <typename T, int L>
__global__ void __launch_bounds__(FastPlan<L>::THREADS)
k_fft_fast(const T* __restrict__ in, T* __restrict__ out, FftParams p, const Ctrl* ctrl, void* const* in_ring) {
  constexpr int SEQ = FastPlan<L>::SEQ, NT = FastPlan<L>::NT, WORDS = FastMap<L>::WORDS, NPEN = 2 * SEQ;
  constexpr int NTH = FastPlan<L>::THREADS, NW = NTH / 32;
  if (ctrl && ctrl->done) return;
  if (in_ring) in = (const T*)in_ring[ctrl->i_local % 4];
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long sbase[NPEN];
  T* buf = (T*)smem_raw;
  Cx<T>* tws = (Cx<T>*)(buf + WORDS);
  const int comp = p.comp0 + blockIdx.y;
  const int type = p.type[comp];
  const int tid = threadIdx.x;
  const long long pen0 = (long long)blockIdx.x * NPEN;
  const T* src = in + (long long)comp * p.NN;
  const long long coff = (long long)comp * p.NN;
  const long long stride = p.axis == 0 ? 1 : (p.axis == 1 ? (long long)p.nnx : (long long)p.nnx * p.nny);
  const int npen = (int)min((long long)NPEN, p.npencil - pen0);
  const int n = p.n, nn = p.nn;
  pencil_bases<T, SEQ>(sbase, p, pen0, tid);
  fast_tw_fill<T, L>(tws, (const Cx<T>*)p.tw, tid, NTH);
  // A full CTA writes every position of its sequences (the fill, then fast_holes); the last
  // CTA of a launch may hold fewer pencils, whose partners must then read as zero.
  const bool full = npen == NPEN;
  if (!full)
    for (int q = tid; q < WORDS; q += NTH) buf[q] = (T)0;
  __syncthreads();
  // global loads in groups of FB per thread before they are placed, so that several are in
  // flight at once
  constexpr int FB = 4;
  // x axis: a warp per pencil row when the rows divide evenly among the warps, else the
  // CTA's rows (consecutive in memory) as one block spread over all threads
  constexpr bool WARP_ROWS = NPEN % NW == 0;
  const float rnn = 1.0f / (float)nn;
  by_type(type, [&](auto ty) {
    constexpr int TY = decltype(ty)::value;
    if (p.axis == 0 && !WARP_ROWS) {
      const T* blk = src + sbase[0];
      const int tot = npen * nn;
      for (int i0 = tid; i0 < tot; i0 += NTH * FB) {
        T v[FB];
        #pragma unroll
        for (int u = 0; u < FB; ++u) {
          const int idx = i0 + NTH * u;
          v[u] = idx < tot ? blk[idx] : (T)0;
        }
        #pragma unroll
        for (int u = 0; u < FB; ++u) {
          const int idx = i0 + NTH * u;
          if (idx < tot) {
            int pb, j;
            row_pos(idx, nn, rnn, pb, j);
            fast_place<T, L>(buf, pb, j, v[u], n, TY, p.inverse);
          }
        }
      }
    } else if (p.axis == 0) {
      const int warp = tid >> 5, lane = tid & 31;
      for (int pb = warp; pb < npen; pb += NW) {
        const T* row = src + sbase[pb];
        for (int j0 = lane; j0 < nn; j0 += 32 * FB) {
          T v[FB];
          #pragma unroll
          for (int u = 0; u < FB; ++u) {
            const int j = j0 + 32 * u;
            v[u] = j < nn ? row[j] : (T)0;
          }
          #pragma unroll
          for (int u = 0; u < FB; ++u) {
            const int j = j0 + 32 * u;
            if (j < nn) fast_place<T, L>(buf, pb, j, v[u], n, TY, p.inverse);
          }
        }
      }
    } else {
      for (int i0 = tid; i0 < NPEN * nn; i0 += NTH * FB) {
        T v[FB];
        #pragma unroll
        for (int u = 0; u < FB; ++u) {
          const int idx = i0 + NTH * u;
          const int pb = idx % NPEN, j = idx / NPEN;
          v[u] = (idx < NPEN * nn && pb < npen) ? src[sbase[pb] + j * stride] : (T)0;
        }
        #pragma unroll
        for (int u = 0; u < FB; ++u) {
          const int idx = i0 + NTH * u;
          const int pb = idx % NPEN, j = idx / NPEN;
          if (idx < NPEN * nn && pb < npen) fast_place<T, L>(buf, pb, j, v[u], n, TY, p.inverse);
        }
      }
    }
    if (full)
      for (int pb = tid; pb < NPEN; pb += NTH) fast_holes<T, L, TY>(buf, pb, n, p.inverse);
  });
  __syncthreads();
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  const int sgn = (p.inverse && quarter) ? 1 : -1;
  const Cx<T>* ph = (const Cx<T>*)p.ph;
  fast_fft<T, L>(buf, tws, sgn, tid / NT, tid % NT, (quarter && !p.inverse) ? ph : nullptr);
  const T sc = sizeof(T) == 4 ? (T)p.fscale : (T)p.scale;
  const T inv_n = sizeof(T) == 4 ? (T)p.finv_n : (T)p.inv_n;
  by_type(type, [&](auto ty) {
    constexpr int TY = decltype(ty)::value;
    auto emit = [&](int pb, int k) {
      const T v = fast_post<T, L>(buf, pb, k, n, TY, p.inverse, sc, ph, inv_n);
      const long long e = coff + sbase[pb] + k * stride;
      if (p.incr) add_to_u<T>(e, v, p);
      else out[e] = v;
    };
    if (p.axis == 0 && !WARP_ROWS) {
      for (int idx = tid; idx < npen * nn; idx += NTH) {
        int pb, k;
        row_pos(idx, nn, rnn, pb, k);
        emit(pb, k);
      }
    } else if (p.axis == 0) {
      const int warp = tid >> 5, lane = tid & 31;
      for (int pb = warp; pb < npen; pb += NW)
        for (int k = lane; k < nn; k += 32) emit(pb, k);
    } else {
      for (int idx = tid; idx < NPEN * nn; idx += NTH) {
        const int pb = idx % NPEN, k = idx / NPEN;
        if (pb < npen) emit(pb, k);
      }
    }
  });
}

// Fused z pass on the register-radix route (same contract as k_fft_z_green).  Five CTAs of
// 256 threads (six of 192) per SM fit its shared memory; the launch bound keeps registers to
// match.
template <typename T, int L>
__global__ void __launch_bounds__(FastPlan<L>::THREADS, FastPlan<L>::MINB)
k_fft_fast_z_green(const T* __restrict__ in, T* __restrict__ out, FftParams p, GreenTables gt, T l0, T m2, T ih2,
                   int scheme, T zscale, const Ctrl* ctrl) {
  constexpr int SEQ = FastPlan<L>::SEQ, NT = FastPlan<L>::NT, WORDS = FastMap<L>::WORDS, NPEN = 2 * SEQ;
  constexpr int NTH = FastPlan<L>::THREADS;
  if (ctrl && ctrl->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ long long sbase[NPEN];
  __shared__ T pxy[NPEN][4];   // per pencil: s_x, c'_x, s_y, c'_y
  T* buf = (T*)smem_raw;
  Cx<T>* tws = (Cx<T>*)(buf + WORDS);
  T* zs = (T*)(tws + L);   // s_z[k], k < nn
  T* zc = zs + p.nn;       // c'_z[k]
  T* spec = zc + p.nn;     // NPEN x nn spectra
  const int comp = p.comp0 + blockIdx.y;
  const int type = p.type[comp];
  const int tid = threadIdx.x;
  const long long pen0 = (long long)blockIdx.x * NPEN;
  const long long coff = (long long)comp * p.NN;
  const long long stride = (long long)p.nnx * p.nny;
  const int npen = (int)min((long long)NPEN, p.npencil - pen0);
  const int n = p.n, nn = p.nn;
  const Cx<T>* ph = (const Cx<T>*)p.ph;
  pencil_bases<T, SEQ>(sbase, p, pen0, tid);
  for (int q = tid; q < NPEN; q += NTH) {
    const long long pen = pen0 + q;
    const int pen32 = pen < p.npencil ? (int)pen : 0;   // z pencils: pen = ix + nnx iy < 2^31
    const int ix = pen32 % p.nnx, iy = pen32 / p.nnx;
    pxy[q][0] = gt_s<T>(gt, comp, 0, ix);
    pxy[q][1] = gt_c<T>(gt, comp, 0, ix);
    pxy[q][2] = gt_s<T>(gt, comp, 1, iy);
    pxy[q][3] = gt_c<T>(gt, comp, 1, iy);
  }
  fast_tw_fill<T, L>(tws, (const Cx<T>*)p.tw, tid, NTH);
  for (int q = tid; q < nn; q += NTH) {
    zs[q] = gt_s<T>(gt, comp, 2, q);
    zc[q] = gt_c<T>(gt, comp, 2, q);
  }
  // see k_fft_fast: only a partial CTA clears its buffer, a full one writes the holes
  const bool full = npen == NPEN;
  if (!full)
    for (int q = tid; q < WORDS; q += NTH) buf[q] = (T)0;
  __syncthreads();
  const bool quarter = (type == T_DCT3 || type == T_DST3);
  const T inv_n = sizeof(T) == 4 ? (T)p.finv_n : (T)p.inv_n;
  by_type(type, [&](auto ty) {
    constexpr int TY = decltype(ty)::value;
    // forward along z
    for (int i0 = tid; i0 < NPEN * nn; i0 += NTH * 4) {
      T v[4];
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = i0 + NTH * u;
        const int pb = idx % NPEN, j = idx / NPEN;
        v[u] = (idx < NPEN * nn && pb < npen) ? in[coff + sbase[pb] + j * stride] : (T)0;
      }
      #pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int idx = i0 + NTH * u;
        const int pb = idx % NPEN, j = idx / NPEN;
        if (idx < NPEN * nn && pb < npen) fast_place<T, L>(buf, pb, j, v[u], n, TY, 0);
      }
    }
    if (full)
      for (int pb = tid; pb < NPEN; pb += NTH) fast_holes<T, L, TY>(buf, pb, n, 0);
    __syncthreads();
    fast_fft<T, L>(buf, tws, -1, tid / NT, tid % NT, quarter ? ph : nullptr);
    // Green multiply into spec
    const T thr = sizeof(T) == 4 ? (T)gt.null_thr_f[comp] : (T)gt.null_thr[comp];
    for (int idx = tid; idx < NPEN * nn; idx += NTH) {
      const int pb = idx % NPEN, k = idx / NPEN;
      T v = (T)0;
      if (pb < npen) {
        v = fast_post<T, L>(buf, pb, k, n, TY, 0, (T)1, ph, inv_n);
        const T sx = pxy[pb][0], cx = pxy[pb][1], sy = pxy[pb][2], cy = pxy[pb][3];
        const T sz = zs[k], cz = zc[k];
        T Sx, Sy, Sz;
        if (scheme == SCHEME_TETRA2) {
          Sx = tetra_S<T>(sx, cy, sy, cx, sz);
          Sy = tetra_S<T>(sy, cz, sz, cy, sx);
          Sz = tetra_S<T>(sz, cx, sx, cz, sy);
        } else {
          Sx = sx * cy * cz;
          Sy = sy * cx * cz;
          Sz = sz * cx * cy;
        }
        const T Sc = comp == 0 ? Sx : (comp == 1 ? Sy : Sz);
        const T a = (l0 * Sc + m2 * (Sx + Sy + Sz)) * ih2;
        v = (a <= thr) ? (T)0 : v / a;
      }
      spec[pb * nn + k] = v;
    }
    __syncthreads();
    // inverse along z
    if (!full) {
      for (int q = tid; q < WORDS; q += NTH) buf[q] = (T)0;
      __syncthreads();
    }
    for (int idx = tid; idx < NPEN * nn; idx += NTH) {
      const int pb = idx % NPEN, j = idx / NPEN;
      if (pb < npen) fast_place<T, L>(buf, pb, j, spec[pb * nn + j], n, TY, 1);
    }
    if (full)
      for (int pb = tid; pb < NPEN; pb += NTH) fast_holes<T, L, TY>(buf, pb, n, 1);
    __syncthreads();
    fast_fft<T, L>(buf, tws, quarter ? 1 : -1, tid / NT, tid % NT, nullptr);
    for (int idx = tid; idx < NPEN * nn; idx += NTH) {
      const int pb = idx % NPEN, k = idx / NPEN;
      if (pb < npen) out[coff + sbase[pb] + k * stride] = fast_post<T, L>(buf, pb, k, n, TY, 1, zscale, ph, inv_n);
    }
  });
}

template <typename K>
static int ensure_smem(K kernel, size_t sm, size_t& done);

// DTT_FFT_GENERIC=1 keeps every length on the generic Stockham kernels (route-agreement
// tests); read at every launch, so it applies to graphs captured after it is set.
static bool generic_only() {
  const char* e = std::getenv("DTT_FFT_GENERIC");
  return e && e[0] == '1';
}

// Register-radix dispatch; returns -1 when L is neither a power of two in 16..2048 nor
// 3 * 2^k in 48..1536 (fused z pass: 16..1024 and 48..768).
template <typename T, int L>
static int launch_fast_L(const T* in, T* out, const FftParams& p, int ncomp, const Ctrl* ctrl, void* const* in_ring,
                         cudaStream_t s) {
  constexpr int NPEN = 2 * FastPlan<L>::SEQ;
  dim3 grd((unsigned)((p.npencil + NPEN - 1) / NPEN), ncomp);
  const size_t sm = fast_smem<T, L>(0);
  static size_t attr = 48 * 1024;
  if (int e = ensure_smem(k_fft_fast<T, L>, sm, attr)) return e;
  k_fft_fast<T, L><<<grd, FastPlan<L>::THREADS, sm, s>>>(in, out, p, ctrl, in_ring);
  return (int)cudaGetLastError();
}

template <typename T, int L>
static int launch_fast_zg_L(const T* in, T* out, const FftParams& p, const GreenTables& gt, T l0, T m2, T ih2,
                            int scheme, T zscale, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  constexpr int NPEN = 2 * FastPlan<L>::SEQ;
  dim3 grd((unsigned)((p.npencil + NPEN - 1) / NPEN), ncomp);
  const size_t sm = fast_smem<T, L>((int)((2 + NPEN) * p.nn * sizeof(T)));
  static size_t attr = 48 * 1024;
  if (int e = ensure_smem(k_fft_fast_z_green<T, L>, sm, attr)) return e;
  k_fft_fast_z_green<T, L><<<grd, FastPlan<L>::THREADS, sm, s>>>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ctrl);
  return (int)cudaGetLastError();
}

template <typename T>
static int launch_fast(const T* in, T* out, const FftParams& p, int ncomp, const Ctrl* ctrl, void* const* in_ring,
                       cudaStream_t s) {
  switch (p.L) {
    case 16: return launch_fast_L<T, 16>(in, out, p, ncomp, ctrl, in_ring, s);
    case 32: return launch_fast_L<T, 32>(in, out, p, ncomp, ctrl, in_ring, s);
    case 64: return launch_fast_L<T, 64>(in, out, p, ncomp, ctrl, in_ring, s);
    case 128: return launch_fast_L<T, 128>(in, out, p, ncomp, ctrl, in_ring, s);
    case 256: return launch_fast_L<T, 256>(in, out, p, ncomp, ctrl, in_ring, s);
    case 512: return launch_fast_L<T, 512>(in, out, p, ncomp, ctrl, in_ring, s);
    case 1024: return launch_fast_L<T, 1024>(in, out, p, ncomp, ctrl, in_ring, s);
    case 2048: return launch_fast_L<T, 2048>(in, out, p, ncomp, ctrl, in_ring, s);
    case 48: return launch_fast_L<T, 48>(in, out, p, ncomp, ctrl, in_ring, s);
    case 96: return launch_fast_L<T, 96>(in, out, p, ncomp, ctrl, in_ring, s);
    case 192: return launch_fast_L<T, 192>(in, out, p, ncomp, ctrl, in_ring, s);
    case 384: return launch_fast_L<T, 384>(in, out, p, ncomp, ctrl, in_ring, s);
    case 768: return launch_fast_L<T, 768>(in, out, p, ncomp, ctrl, in_ring, s);
    case 1536: return launch_fast_L<T, 1536>(in, out, p, ncomp, ctrl, in_ring, s);
    default: return -1;
  }
}

template <typename T>
static int launch_fast_zg(const T* in, T* out, const FftParams& p, const GreenTables& gt, T l0, T m2, T ih2,
                          int scheme, T zscale, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  switch (p.L) {
    case 16: return launch_fast_zg_L<T, 16>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 32: return launch_fast_zg_L<T, 32>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 64: return launch_fast_zg_L<T, 64>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 128: return launch_fast_zg_L<T, 128>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 256: return launch_fast_zg_L<T, 256>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 512: return launch_fast_zg_L<T, 512>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 1024: return launch_fast_zg_L<T, 1024>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 48: return launch_fast_zg_L<T, 48>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 96: return launch_fast_zg_L<T, 96>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 192: return launch_fast_zg_L<T, 192>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 384: return launch_fast_zg_L<T, 384>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    case 768: return launch_fast_zg_L<T, 768>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    default: return -1;
  }
}

template <typename T>
int fft_pb(int L) {
  // pairs per CTA: two buffers of PB * L complex values within ~100 KB of shared memory
  const int bytes = 2 * L * (int)sizeof(Cx<T>);
  int pb = 102400 / bytes;
  if (pb >= 8) return 8;
  if (pb >= 4) return 4;
  if (pb >= 2) return 2;
  return pb >= 1 ? 1 : 0;
}

template <typename K>
static int ensure_smem(K kernel, size_t sm, size_t& done) {
  if (sm <= done) return 0;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return (int)e;
  done = sm;
  return 0;
}

template <typename T, int PB>
static int launch_fft_pb(const T* in, T* out, const FftParams& p, int ncomp, const Ctrl* ctrl, void* const* in_ring,
                         cudaStream_t s) {
  dim3 grd((unsigned)((p.npencil + 2 * PB - 1) / (2 * PB)), ncomp);
  const size_t sm = fft_smem_base<T, PB>(p.L);
  static size_t attr = 48 * 1024;
  if (int e = ensure_smem(k_fft_axis<T, PB>, sm, attr)) return e;
  k_fft_axis<T, PB><<<grd, 256, sm, s>>>(in, out, p, ctrl, in_ring);
  return (int)cudaGetLastError();
}

template <typename T, int PB>
static int launch_zg_pb(const T* in, T* out, const FftParams& p, const GreenTables& gt, double lam0, double mu0,
                        int scheme, double h, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  dim3 grd((unsigned)((p.npencil + 2 * PB - 1) / (2 * PB)), ncomp);
  const size_t sm = fft_smem_base<T, PB>(p.L) + (size_t)2 * p.nn * sizeof(T);
  static size_t attr = 48 * 1024;
  if (int e = ensure_smem(k_fft_z_green<T, PB>, sm, attr)) return e;
  const T l0 = (T)lam0, m2 = (T)(2.0 * mu0), ih2 = (T)(4.0 / (h * h));
  const T zscale = (T)((p.L == p.n) ? 1.0 / p.n : 2.0 / p.n);   // Hartley 1/n, DCT1 / DST1 2/n
  k_fft_z_green<T, PB><<<grd, 256, sm, s>>>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ctrl);
  return (int)cudaGetLastError();
}

template <typename T>
int launch_fft_z_green(const T* in, T* out, const FftParams& p, const GreenTables& gt, double lam0, double mu0,
                       int scheme, double h, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  if (!p.generic && !generic_only()) {
    const T l0 = (T)lam0, m2 = (T)(2.0 * mu0), ih2 = (T)(4.0 / (h * h));
    const T zscale = (T)((p.L == p.n) ? 1.0 / p.n : 2.0 / p.n);
    const int r = launch_fast_zg<T>(in, out, p, gt, l0, m2, ih2, scheme, zscale, ncomp, ctrl, s);
    if (r >= 0) return r;
  }
  switch (fft_pb<T>(p.L)) {
    case 8: return launch_zg_pb<T, 8>(in, out, p, gt, lam0, mu0, scheme, h, ncomp, ctrl, s);
    case 4: return launch_zg_pb<T, 4>(in, out, p, gt, lam0, mu0, scheme, h, ncomp, ctrl, s);
    case 2: return launch_zg_pb<T, 2>(in, out, p, gt, lam0, mu0, scheme, h, ncomp, ctrl, s);
    case 1: return launch_zg_pb<T, 1>(in, out, p, gt, lam0, mu0, scheme, h, ncomp, ctrl, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template <typename T>
int launch_fft_axis(const T* in, T* out, const FftParams& p, int ncomp, const Ctrl* ctrl, void* const* in_ring,
                    cudaStream_t s) {
  if (!p.generic && !generic_only()) {
    const int r = launch_fast<T>(in, out, p, ncomp, ctrl, in_ring, s);
    if (r >= 0) return r;
  }
  switch (fft_pb<T>(p.L)) {
    case 8: return launch_fft_pb<T, 8>(in, out, p, ncomp, ctrl, in_ring, s);
    case 4: return launch_fft_pb<T, 4>(in, out, p, ncomp, ctrl, in_ring, s);
    case 2: return launch_fft_pb<T, 2>(in, out, p, ncomp, ctrl, in_ring, s);
    case 1: return launch_fft_pb<T, 1>(in, out, p, ncomp, ctrl, in_ring, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

template int launch_fft_axis<double>(const double*, double*, const FftParams&, int, const Ctrl*, void* const*, cudaStream_t);
template int launch_fft_axis<float>(const float*, float*, const FftParams&, int, const Ctrl*, void* const*, cudaStream_t);
template int launch_fft_z_green<double>(const double*, double*, const FftParams&, const GreenTables&, double, double, int, double, int, const Ctrl*, cudaStream_t);
template int launch_fft_z_green<float>(const float*, float*, const FftParams&, const GreenTables&, double, double, int, double, int, const Ctrl*, cudaStream_t);
template int fft_pb<double>(int);
template int fft_pb<float>(int);

}  // namespace dtt
