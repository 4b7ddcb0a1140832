// Warp-register DTT passes of the mixed-precision Green step (FP32).
//
// The Green step (Section 3.2.2, Tables 2-3, Eq. 7) is five sweeps over the three
// components: forward DTT along x and along y, the fused forward z DTT + Green multiply +
// inverse z DTT, inverse DTT along y and along x (the last one adds its result to u~).
// Here every sweep reads contiguous rows along its own axis and hands the next sweep
// contiguous rows along the next axis: each of the first four writes its result
// transposed, through a shared-memory tile, so that no sweep gathers strided pencils.
//
//   sweep  reads rows of           row length   writes
//   fx     natural [c][z][y][x]    nx           T1 [c][z][kx][y]
//   fy     T1                      ny           T2 [c][kx][ky][z]
//   zg     T2                      nz           T3 [c][z][kx][ky]   (Green multiply inside)
//   iy     T3                      ny           T4 [c][z][y][kx]
//   ix     T4                      nx           natural (or u~ += result, step = result)
//
// One DTT of a pair of real rows (a, b) is one complex FFT of length L = 2n of the
// extension of z = a + i b (the extensions of Table 3 per transform type, as in the
// shared-memory Stockham kernels).  A warp owns P = 32 / R such pairs (L = 32 R) and takes
// each FFT in two register stages with one shared-memory transpose between them:
//   stage 1: lane l holds z_(l + 32 m), m < R, and takes the R-point DFT over m in
//            registers, then multiplies by w_L^(l k1);
//   stage 2: lane t = q R + k1 holds the 32 values of sequence q at k1 and takes the
//            32-point DFT over l in registers, giving X_(k1 + R k2).
// R is 2, 3, 4, 6, 8, 12, 16, 24 or 32 (n = 32 ... 512 voxels along every axis of the grid,
// none periodic); 32 - P R lanes idle in stage 2 (8 for R = 12 and 24, 2 for R = 3 and 6).
// The butterflies are fully unrolled with compile-time twiddles; only the stage-1
// twiddles w_L^(l k1) come from a small [R][32] table.  No block-wide barrier is needed
// until the tile of transposed results is written out.
#include <cstdint>
#include <type_traits>

#include "dtt_internal.cuh"

namespace dtt {

namespace {

// ---- compile-time trigonometry: cos and sin of 2 pi m / N ------------------------------
constexpr double kPi = 3.14159265358979323846;
constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 24; ++k) {
    term *= -x * x / ((double)(2 * k - 1) * (double)(2 * k));
    sum += term;
  }
  return sum;
}
constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 24; ++k) {
    term *= -x * x / ((double)(2 * k) * (double)(2 * k + 1));
    sum += term;
  }
  return sum;
}
// quadrant q and the angle a in [0, pi/2) with 2 pi m / N = q pi / 2 + a
constexpr double cos2pi(long long m, long long N) {
  m %= N;
  if (m < 0) m += N;
  const long long q = (4 * m) / N, r = 4 * m - q * N;
  if (r == 0) return q == 0 ? 1.0 : (q == 2 ? -1.0 : 0.0);
  const double a = (kPi / 2) * (double)r / (double)N;
  const double c = taylor_cos(a), s = taylor_sin(a);
  return q == 0 ? c : (q == 1 ? -s : (q == 2 ? -c : s));
}
constexpr double sin2pi(long long m, long long N) {
  m %= N;
  if (m < 0) m += N;
  const long long q = (4 * m) / N, r = 4 * m - q * N;
  if (r == 0) return q == 1 ? 1.0 : (q == 3 ? -1.0 : 0.0);
  const double a = (kPi / 2) * (double)r / (double)N;
  const double c = taylor_cos(a), s = taylor_sin(a);
  return q == 0 ? s : (q == 1 ? c : (q == 2 ? -s : -c));
}

template <int B, int E, typename F>
__device__ __forceinline__ void sfor(F&& f) {
  if constexpr (B < E) {
    f(std::integral_constant<int, B>());
    sfor<B + 1, E>(f);
  }
}

struct C2 {
  float x, y;
};

__device__ __forceinline__ C2 cadd(C2 a, C2 b) { return C2{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ C2 csub(C2 a, C2 b) { return C2{a.x - b.x, a.y - b.y}; }

// v * e^(S 2 pi i M / N), the quarter turns as swaps and negations
template <int N, int M, int S>
__device__ __forceinline__ C2 twmul(C2 v) {
  constexpr int mm = ((M % N) + N) % N;
  if constexpr (mm == 0) {
    return v;
  } else if constexpr (2 * mm == N) {
    return C2{-v.x, -v.y};
  } else if constexpr (4 * mm == N) {
    return S > 0 ? C2{-v.y, v.x} : C2{v.y, -v.x};
  } else if constexpr (4 * mm == 3 * N) {
    return S > 0 ? C2{v.y, -v.x} : C2{-v.y, v.x};
  } else {
    constexpr float c = (float)cos2pi(mm, N);
    constexpr float s = (float)((double)S * sin2pi(mm, N));
    return C2{v.x * c - v.y * s, v.x * s + v.y * c};
  }
}

// In-place DFT of N values in registers, natural order in and out:
//   v_k <- sum_j v_j e^(S 2 pi i j k / N).
// Composite N = N1 N2 (N1 = 4, 2 or 3): N2 DFTs of N1 points over j = N2 j1 + j2, the
// twiddles e^(S 2 pi i j2 k1 / N), then N1 DFTs of N2 points, output k = k1 + N1 k2.
template <int N, int S>
struct Dft {
  static constexpr int N1 = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
  static constexpr int N2 = N / N1;
  __device__ __forceinline__ static void run(C2* v) {
    C2 w[N];
    sfor<0, N2>([&](auto j2c) {
      constexpr int j2 = decltype(j2c)::value;
      C2 t[N1];
      sfor<0, N1>([&](auto j1c) {
        constexpr int j1 = decltype(j1c)::value;
        t[j1] = v[N2 * j1 + j2];
      });
      Dft<N1, S>::run(t);
      sfor<0, N1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        w[j2 * N1 + k1] = twmul<N, j2 * k1, S>(t[k1]);
      });
    });
    sfor<0, N1>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      C2 t[N2];
      sfor<0, N2>([&](auto j2c) {
        constexpr int j2 = decltype(j2c)::value;
        t[j2] = w[j2 * N1 + k1];
      });
      Dft<N2, S>::run(t);
      sfor<0, N2>([&](auto k2c) {
        constexpr int k2 = decltype(k2c)::value;
        v[k1 + N1 * k2] = t[k2];
      });
    });
  }
};
template <int S>
struct Dft<1, S> {
  __device__ __forceinline__ static void run(C2*) {}
};
template <int S>
struct Dft<2, S> {
  __device__ __forceinline__ static void run(C2* v) {
    const C2 a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  }
};
template <int S>
struct Dft<3, S> {
  __device__ __forceinline__ static void run(C2* v) {
    // y1,2 = x0 - (x1 + x2) / 2 +- i S (sqrt 3 / 2) (x1 - x2)
    constexpr float h = 0.8660254037844386f;
    const C2 s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const C2 m = C2{v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y};
    const C2 r = S > 0 ? C2{-h * d.y, h * d.x} : C2{h * d.y, -h * d.x};
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, r);
    v[2] = csub(m, r);
  }
};
template <int S>
struct Dft<4, S> {
  __device__ __forceinline__ static void run(C2* v) {
    const C2 a = cadd(v[0], v[2]), b = csub(v[0], v[2]);
    const C2 c = cadd(v[1], v[3]), d = csub(v[1], v[3]);
    const C2 id = S > 0 ? C2{-d.y, d.x} : C2{d.y, -d.x};   // i S d
    v[0] = cadd(a, c);
    v[2] = csub(a, c);
    v[1] = cadd(b, id);
    v[3] = csub(b, id);
  }
};

// ---- two DFTs at once in the lanes of packed FP32x2 registers ----------------------------
// P2 holds the same position of two independent sequences: re = (a.re, b.re), im =
// (a.im, b.im); every butterfly and twiddle below is one packed instruction per part.
struct P2 {
  float2 re, im;
};
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  float2 r;
  asm("{ .reg .b64 ra, rb, rr; mov.b64 ra, {%2, %3}; mov.b64 rb, {%4, %5}; sub.rn.f32x2 rr, ra, rb; mov.b64 {%0, %1}, rr; }"
      : "=f"(r.x), "=f"(r.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2c(float v) { return make_float2(v, v); }
__device__ __forceinline__ P2 padd(P2 a, P2 b) { return P2{f2add(a.re, b.re), f2add(a.im, b.im)}; }
__device__ __forceinline__ P2 psub(P2 a, P2 b) { return P2{f2sub(a.re, b.re), f2sub(a.im, b.im)}; }
// a + i T b (T = +1 or -1)
template <int T>
__device__ __forceinline__ P2 padd_i(P2 a, P2 b) {
  return T > 0 ? P2{f2sub(a.re, b.im), f2add(a.im, b.re)} : P2{f2add(a.re, b.im), f2sub(a.im, b.re)};
}

// v * e^(S 2 pi i M / N) in both lanes
template <int N, int M, int S>
__device__ __forceinline__ P2 ptwmul(P2 v) {
  constexpr int mm = ((M % N) + N) % N;
  if constexpr (mm == 0) {
    return v;
  } else if constexpr (2 * mm == N) {
    return P2{f2mul(v.re, f2c(-1.f)), f2mul(v.im, f2c(-1.f))};
  } else if constexpr (4 * mm == N) {   // i S v
    return S > 0 ? P2{f2mul(v.im, f2c(-1.f)), v.re} : P2{v.im, f2mul(v.re, f2c(-1.f))};
  } else if constexpr (4 * mm == 3 * N) {   // -i S v
    return S > 0 ? P2{v.im, f2mul(v.re, f2c(-1.f))} : P2{f2mul(v.im, f2c(-1.f)), v.re};
  } else {
    constexpr float c = (float)cos2pi(mm, N);
    constexpr float s = (float)((double)S * sin2pi(mm, N));
    return P2{f2fma(v.im, f2c(-s), f2mul(v.re, f2c(c))), f2fma(v.im, f2c(c), f2mul(v.re, f2c(s)))};
  }
}

// Two in-place DFTs of N values (same plan as Dft, on packed pairs).
template <int N, int S>
struct Dft2 {
  static constexpr int N1 = (N % 4 == 0) ? 4 : ((N % 2 == 0) ? 2 : 3);
  static constexpr int N2 = N / N1;
  __device__ __forceinline__ static void run(P2* v) {
    P2 w[N];
    sfor<0, N2>([&](auto j2c) {
      constexpr int j2 = decltype(j2c)::value;
      P2 t[N1];
      sfor<0, N1>([&](auto j1c) {
        constexpr int j1 = decltype(j1c)::value;
        t[j1] = v[N2 * j1 + j2];
      });
      Dft2<N1, S>::run(t);
      sfor<0, N1>([&](auto k1c) {
        constexpr int k1 = decltype(k1c)::value;
        w[j2 * N1 + k1] = ptwmul<N, j2 * k1, S>(t[k1]);
      });
    });
    sfor<0, N1>([&](auto k1c) {
      constexpr int k1 = decltype(k1c)::value;
      P2 t[N2];
      sfor<0, N2>([&](auto j2c) {
        constexpr int j2 = decltype(j2c)::value;
        t[j2] = w[j2 * N1 + k1];
      });
      Dft2<N2, S>::run(t);
      sfor<0, N2>([&](auto k2c) {
        constexpr int k2 = decltype(k2c)::value;
        v[k1 + N1 * k2] = t[k2];
      });
    });
  }
};
template <int S>
struct Dft2<1, S> {
  __device__ __forceinline__ static void run(P2*) {}
};
template <int S>
struct Dft2<2, S> {
  __device__ __forceinline__ static void run(P2* v) {
    const P2 a = v[0], b = v[1];
    v[0] = padd(a, b);
    v[1] = psub(a, b);
  }
};
template <int S>
struct Dft2<3, S> {
  __device__ __forceinline__ static void run(P2* v) {
    constexpr float h = 0.8660254037844386f;
    const P2 s = padd(v[1], v[2]), d = psub(v[1], v[2]);
    const P2 m = P2{f2fma(s.re, f2c(-0.5f), v[0].re), f2fma(s.im, f2c(-0.5f), v[0].im)};
    // m +- i S h d
    v[0] = padd(v[0], s);
    v[1] = P2{f2fma(d.im, f2c(-S * h), m.re), f2fma(d.re, f2c(S * h), m.im)};
    v[2] = P2{f2fma(d.im, f2c(S * h), m.re), f2fma(d.re, f2c(-S * h), m.im)};
  }
};
template <int S>
struct Dft2<4, S> {
  __device__ __forceinline__ static void run(P2* v) {
    const P2 a = padd(v[0], v[2]), b = psub(v[0], v[2]);
    const P2 c = padd(v[1], v[3]), d = psub(v[1], v[3]);
    v[0] = padd(a, c);
    v[2] = psub(a, c);
    v[1] = padd_i<S>(b, d);
    v[3] = padd_i<-S>(b, d);
  }
};

// One DFT of N values (N even), natural order, of which the first NK outputs are formed:
// the even- and odd-indexed halves run as the two lanes of one packed DFT of N / 2, then
// X_k = E_k + w^k O_k and X_(k + N/2) = E_k - w^k O_k with w = e^(S 2 pi i / N).
template <int N, int S, int NK = N>
__device__ __forceinline__ void dft_split(C2* v) {
  if constexpr (N % 2 != 0) {
    Dft<N, S>::run(v);
  } else {
    constexpr int H = N / 2;
    P2 t[H];
#pragma unroll
    for (int m = 0; m < H; ++m) t[m] = P2{make_float2(v[2 * m].x, v[2 * m + 1].x), make_float2(v[2 * m].y, v[2 * m + 1].y)};
    Dft2<H, S>::run(t);
    sfor<0, H>([&](auto kc) {
      constexpr int k = decltype(kc)::value;
      const C2 e = C2{t[k].re.x, t[k].im.x};
      const C2 o = twmul<N, k, S>(C2{t[k].re.y, t[k].im.y});
      if constexpr (k < NK) v[k] = cadd(e, o);
      if constexpr (k + H < NK) v[k + H] = csub(e, o);
    });
  }
}

// ---- plan of one pass --------------------------------------------------------------
template <int R>
struct WPlan {
  static constexpr int L = 32 * R;               // FFT length (2n)
  static constexpr int P = R >= 32 ? 1 : 32 / R;   // sequences (row pairs) per warp
  static constexpr int Q = P * R;                // lanes busy in stage 2
  static constexpr int QS = L + R;               // stride of a sequence in the fill layout
  static constexpr int SW = Q * 33;              // words of each scratch array (re, im)
  static constexpr int NI = R / 2 + 1;           // 32-wide chunks of one row (len <= 16 R + 1)
  static_assert(SW >= (P - 1) * QS + L, "scratch too small for the fill layout");
};

// Value pair (va, vb) of input position j into the extended sequence (re / im arrays of
// one sequence), per transform type; the inverse quarter-wave types take the spectrum
// extended as X_(2n-1-k) = +-X_k.
template <int TY, bool INV>
__device__ __forceinline__ void wplace(float* qr, float* qi, int j, float va, float vb, int n) {
  constexpr bool quarter = (TY == T_DCT3 || TY == T_DST3);
  auto S = [&](int pos, float sa, float sb) {
    qr[pos] = sa;
    qi[pos] = sb;
  };
  if constexpr (INV && quarter) {
    if (j < n) {
      S(j, va, vb);
      if constexpr (TY == T_DCT3) S(2 * n - 1 - j, va, vb);
      else S(2 * n - 1 - j, -va, -vb);
    }
  } else if constexpr (TY == T_DCT1) {
    S(j, va, vb);
    if (j >= 1 && j <= n - 1) S(2 * n - j, va, vb);
  } else if constexpr (TY == T_DST1) {
    if (j >= 1 && j <= n - 1) {
      S(j, va, vb);
      S(2 * n - j, -va, -vb);
    }
  } else if constexpr (TY == T_DCT3) {
    if (j <= n - 1) {
      S(j, va, vb);
      if (j >= 1) S(2 * n - j, -va, -vb);
    }
  } else {   // T_DST3 forward
    if (j >= 1) {
      S(j, va, vb);
      if (j <= n - 1) S(2 * n - j, va, vb);
    }
  }
}

// Positions of the extended sequence that wplace leaves unwritten (set to zero).
template <int TY, bool INV>
__device__ __forceinline__ void wholes(float* qr, float* qi, int n) {
  if constexpr (TY == T_DST1) {
    qr[0] = 0.f;
    qi[0] = 0.f;
    qr[n] = 0.f;
    qi[n] = 0.f;
  } else if constexpr (TY == T_DCT3 && !INV) {
    qr[n] = 0.f;
    qi[n] = 0.f;
  } else if constexpr (TY == T_DST3 && !INV) {
    qr[0] = 0.f;
    qi[0] = 0.f;
  }
}

// Transform values of the two rows at output position k from the FFT value X = X_k:
// forward, or inverse of a non-quarter type (scaled by sc); inverse quarter-wave types
// read e = X e^(+i pi k / 2n) and scale by 1/n.
template <int TY, bool INV>
__device__ __forceinline__ void wpost(C2 X, int k, int n, float sc, float inv_n, const float2* ph, float& va,
                                      float& vb) {
  constexpr bool quarter = (TY == T_DCT3 || TY == T_DST3);
  if constexpr (INV && quarter) {
    const float2 w = __ldg(ph + k);   // e^(-i pi k / 2n); its conjugate is applied
    const float ex = X.x * w.x + X.y * w.y, ey = X.y * w.x - X.x * w.y;
    if constexpr (TY == T_DCT3) {
      const bool ok = k <= n - 1;
      va = ok ? ex * inv_n : 0.f;
      vb = ok ? ey * inv_n : 0.f;
    } else {
      const bool ok = k >= 1;
      va = ok ? ey * inv_n : 0.f;
      vb = ok ? -ex * inv_n : 0.f;
    }
  } else {
    const float hs = 0.5f * sc;
    if constexpr (TY == T_DCT1) {
      va = hs * X.x;
      vb = hs * X.y;
    } else if constexpr (TY == T_DST1) {
      const bool ok = k >= 1 && k <= n - 1;
      va = ok ? -hs * X.y : 0.f;
      vb = ok ? hs * X.x : 0.f;
    } else if constexpr (TY == T_DCT3) {
      const bool ok = k <= n - 1;
      va = ok ? hs * X.x : 0.f;
      vb = ok ? hs * X.y : 0.f;
    } else {
      const bool ok = k <= n - 1;
      va = ok ? -hs * X.y : 0.f;
      vb = ok ? hs * X.x : 0.f;
    }
  }
}

// Stage 1 and stage 2 of the P FFTs of one warp, from the fill layout in (sr, si) (with
// the quarter-wave modulation of forward DCT3 / DST3 applied on the way in).  On return
// lane t = q R + k1 (t < Q) holds X[k2] = X_(k1 + R k2) of sequence q for k2 < NK; the
// scratch may be overwritten.
template <int R, int S, bool MOD, int NK>
__device__ __forceinline__ void wfft(float* sr, float* si, const float2* tw1, const float2* ph, int lane, C2* X) {
  using PL = WPlan<R>;
  constexpr int P = PL::P, Q = PL::Q;
  __syncwarp();
  C2 z[P][R];
#pragma unroll
  for (int q = 0; q < P; ++q) {
#pragma unroll
    for (int m = 0; m < R; ++m) {
      const int pos = q * PL::QS + lane + 32 * m;
      z[q][m] = C2{sr[pos], si[pos]};
      if constexpr (MOD) {
        const float2 w = __ldg(ph + lane + 32 * m);
        const C2 v = z[q][m];
        z[q][m] = C2{v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x};
      }
    }
  }
  __syncwarp();
#pragma unroll
  for (int q = 0; q < P; ++q) dft_split<R, S>(z[q]);
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) {
    float2 w = __ldg(tw1 + k1 * 32 + lane);   // e^(-2 pi i lane k1 / L)
    if constexpr (S > 0) w.y = -w.y;
#pragma unroll
    for (int q = 0; q < P; ++q) {
      const C2 v = z[q][k1];
      z[q][k1] = C2{v.x * w.x - v.y * w.y, v.x * w.y + v.y * w.x};
    }
  }
#pragma unroll
  for (int q = 0; q < P; ++q)
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const int pos = (q * R + k1) * 33 + lane;
      sr[pos] = z[q][k1].x;
      si[pos] = z[q][k1].y;
    }
  __syncwarp();
  const int t = lane < Q ? lane : Q - 1;
  C2 x[32];
#pragma unroll
  for (int l = 0; l < 32; ++l) x[l] = C2{sr[t * 33 + l], si[t * 33 + l]};
  __syncwarp();
  dft_split<32, S, NK>(x);
#pragma unroll
  for (int k2 = 0; k2 < NK; ++k2) X[k2] = x[k2];
}

// Loads the P row pairs of this warp (rows 2 (p0 + q), + 1 of the CTA, zero beyond
// nvalid) and writes their extended sequences into the fill layout.
template <int R, int TY, bool INV>
__device__ __forceinline__ void wfill(float* sr, float* si, const float* __restrict__ src, long long row_stride,
                                      int p0, int nvalid, int len, int n, int lane) {
  using PL = WPlan<R>;
  constexpr int P = PL::P, NI = PL::NI;
  float a[P][NI], b[P][NI];
#pragma unroll
  for (int q = 0; q < P; ++q) {
    const int ra = 2 * (p0 + q);
    const bool oka = ra < nvalid, okb = ra + 1 < nvalid;
    const float* pa = src + (long long)ra * row_stride;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int j = lane + 32 * i;
      a[q][i] = (oka && j < len) ? pa[j] : 0.f;
      b[q][i] = (okb && j < len) ? pa[row_stride + j] : 0.f;
    }
  }
#pragma unroll
  for (int q = 0; q < P; ++q) {
    float* qr = sr + q * PL::QS;
    float* qi = si + q * PL::QS;
#pragma unroll
    for (int i = 0; i < NI; ++i) {
      const int j = lane + 32 * i;
      if (j < len) wplace<TY, INV>(qr, qi, j, a[q][i], b[q][i], n);
    }
    if (lane == 0) wholes<TY, INV>(qr, qi, n);
  }
}

}  // namespace

// MODE 0: transposed output through the tile; MODE 2: row output (or increment into u~).
// TY, INV: transform type of the covered components and direction (one FFT body per kernel)
template <int R, int NW, int MODE, int TY, bool INV>
__global__ void __launch_bounds__(NW * 32, 16 / NW)
k_wfft(WfftPass p, const Ctrl* ctrl) {
  using PL = WPlan<R>;
  constexpr int P = PL::P, Q = PL::Q, RPC = 2 * P * NW, RPCP = RPC + 1, NK = 17;
  if (ctrl && ctrl->done) return;
  const float* in = p.in_ring ? (const float*)p.in_ring[ctrl->i_local % 4] : p.in;
  extern __shared__ __align__(16) float wsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sr = wsm + warp * 2 * PL::SW;
  float* si = sr + PL::SW;
  float* tile = wsm + NW * 2 * PL::SW;
  const int comp = p.comp0 + blockIdx.z;
  const int row0 = blockIdx.x * p.rpt;
  const int nvalid = min(p.rpt, p.nrows - row0);
  const long long ib = (long long)comp * p.NN + (long long)blockIdx.y * p.in_outer + (long long)row0 * p.in_row;
  const int n = p.n, len = p.len;
  const int LENP = len | 1;   // row stride of the MODE 2 tile (odd: lanes of two rows spread)
  const int p0 = warp * P;
  const bool busy = 2 * p0 < nvalid;
  {
    constexpr bool quarter = (TY == T_DCT3 || TY == T_DST3);
    if (busy) {
      C2 X[NK];
      if constexpr (INV) {
        wfill<R, TY, true>(sr, si, in + ib, p.in_row, p0, nvalid, len, n, lane);
        wfft<R, quarter ? 1 : -1, false, NK>(sr, si, p.tw1, p.ph, lane, X);
      } else {
        wfill<R, TY, false>(sr, si, in + ib, p.in_row, p0, nvalid, len, n, lane);
        wfft<R, -1, quarter, NK>(sr, si, p.tw1, p.ph, lane, X);
      }
      if (lane < Q) {
        const int q = lane / R, k1 = lane - q * R;
        const int ra = 2 * (p0 + q);
#pragma unroll
        for (int k2 = 0; k2 < NK; ++k2) {
          const int k = k1 + R * k2;
          if (k < len) {
            float va, vb;
            wpost<TY, INV>(X[k2], k, n, p.sc, p.inv_n, p.ph, va, vb);
            if constexpr (MODE == 0) {
              tile[k * RPCP + ra] = va;
              tile[k * RPCP + ra + 1] = vb;
            } else {
              tile[ra * LENP + k] = va;
              tile[(ra + 1) * LENP + k] = vb;
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if constexpr (MODE == 0) {
    const long long ob = (long long)comp * p.NN + (long long)blockIdx.y * p.out_outer + row0;
    for (int e = threadIdx.x; e < len * RPC; e += NW * 32) {
      const int k = e / RPC, r = e - k * RPC;
      if (r < nvalid) p.out[ob + (long long)k * p.out_k + r] = tile[k * RPCP + r];
    }
  } else if (p.in_row == len) {
    // the CTA's rows are one contiguous block: coalesced read-modify-write of u~ (or a
    // plain store), all loads of a thread's group issued before its stores
    const int tot = nvalid * len;
    constexpr int U = 8;
    for (int e0 = threadIdx.x; e0 < tot; e0 += NW * 32 * U) {
      float v[U], h[U], l[U];
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NW * 32;
        const int r = e / len, k = e - r * len;
        v[u] = e < tot ? tile[r * LENP + k] : 0.f;
        if (p.uhi && e < tot) {
          h[u] = p.uhi[ib + e];
          l[u] = p.ulo[ib + e];
        }
      }
#pragma unroll
      for (int u = 0; u < U; ++u) {
        const int e = e0 + u * NW * 32;
        if (e >= tot) break;
        if (p.uhi) {
          ff_add(h[u], l[u], v[u]);
          p.uhi[ib + e] = h[u];
          p.ulo[ib + e] = l[u];
          if (p.step) p.step[ib + e] = v[u];
        } else {
          p.out[ib + e] = v[u];
        }
      }
    }
  } else {
    for (int e = threadIdx.x; e < nvalid * len; e += NW * 32) {
      const int r = e / len, k = e - r * len;
      const long long ea = ib + (long long)r * p.in_row + k;
      const float v = tile[r * LENP + k];
      if (p.uhi) {
        float h = p.uhi[ea], l = p.ulo[ea];
        ff_add(h, l, v);
        p.uhi[ea] = h;
        p.ulo[ea] = l;
        if (p.step) p.step[ea] = v;
      } else {
        p.out[ea] = v;
      }
    }
  }
}

// Fused z pass: forward z DTT of the rows (c, kx, ky), Green multiply (the Paux symbol
// of Section 3.2.3 with the TETRA2 / HEX1 S_j), inverse z DTT, written transposed.
// TY: the transform type of every component the launch covers (one body per type keeps
// the unrolled forward and inverse FFTs within the instruction cache)
template <int R, int NW, int TY>
__global__ void __launch_bounds__(NW * 32, 16 / NW)
k_wfft_zg(WfftPass p, GreenTables gt, float l0, float m2, float ih2, int scheme, const Ctrl* ctrl) {
  using PL = WPlan<R>;
  constexpr int P = PL::P, Q = PL::Q, RPC = 2 * P * NW, RPCP = RPC + 1, NK = 17;
  if (ctrl && ctrl->done) return;
  extern __shared__ __align__(16) float wsm[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float* sr = wsm + warp * 2 * PL::SW;
  float* si = sr + PL::SW;
  float* tile = wsm + NW * 2 * PL::SW;
  const int comp = p.comp0 + blockIdx.z;
  const int kx = blockIdx.y;
  const int row0 = blockIdx.x * p.rpt;
  const int nvalid = min(p.rpt, p.nrows - row0);
  const long long ib = (long long)comp * p.NN + (long long)kx * p.in_outer + (long long)row0 * p.in_row;
  const int n = p.n, len = p.len;
  const int p0 = warp * P;
  const bool busy = 2 * p0 < nvalid;
  const float sx = gt.sf[comp][0][kx], cx = gt.cpf[comp][0][kx];
  const float thr = gt.null_thr_f[comp];
  {
    constexpr bool quarter = (TY == T_DCT3 || TY == T_DST3);
    if (busy) {
      C2 X[NK];
      wfill<R, TY, false>(sr, si, p.in + ib, p.in_row, p0, nvalid, len, n, lane);
      wfft<R, -1, quarter, NK>(sr, si, p.tw1, p.ph, lane, X);
      // Green multiply, then the spectrum into the fill layout of the inverse
      const int q = lane / R, k1 = lane - q * R;
      const int ra = 2 * (p0 + q);
      const int kya = min(row0 + ra, p.nrows - 1), kyb = min(row0 + ra + 1, p.nrows - 1);
      const float sya = gt.sf[comp][1][kya], cya = gt.cpf[comp][1][kya];
      const float syb = gt.sf[comp][1][kyb], cyb = gt.cpf[comp][1][kyb];
      float* qr = sr + q * PL::QS;
      float* qi = si + q * PL::QS;
      // The symbol a_c = (lambda0 S_c + 2 mu0 (S_x + S_y + S_z)) 4 / h^2 with, for TETRA2,
      // S_x / 4 = s_x c'_y + s_z (s_y - s_x), S_y / 4 = s_y c'_z + s_x (s_z - s_y),
      // S_z / 4 = s_z c'_x + s_y (s_x - s_z), each difference s_b - s_a taken as c'_a - c'_b
      // when s_a + s_b >= 1 (no cancellation near the checkerboard mode); HEX1:
      // S_x / 4 = s_x c'_y c'_z and cyclically.  The parts fixed by the row (k_x, k_y) are
      // formed once; the z position k adds s_z, c'_z.
      auto dif = [](float sa, float sb, float ca, float cb) { return (sa + sb < 1.f) ? (sb - sa) : (ca - cb); };
      const float dxya = dif(sx, sya, cx, cya), dxyb = dif(sx, syb, cx, cyb);
      auto symbol = [&](float sy, float cy, float dxy, float sz, float cz, float dzx) {
        float Sx, Sy, Sz;
        if (scheme == SCHEME_TETRA2) {
          Sx = sx * cy + sz * dxy;
          Sy = sy * cz + sx * dif(sy, sz, cy, cz);
          Sz = sz * cx + sy * dzx;
        } else {
          Sx = sx * cy * cz;
          Sy = sy * cx * cz;
          Sz = sz * cx * cy;
        }
        const float Sc = comp == 0 ? Sx : (comp == 1 ? Sy : Sz);
        return (l0 * Sc + m2 * (Sx + Sy + Sz)) * ih2;
      };
      if (lane < Q) {
#pragma unroll
        for (int k2 = 0; k2 < NK; ++k2) {
          const int k = k1 + R * k2;
          if (k < len) {
            float va, vb;
            wpost<TY, false>(X[k2], k, n, 1.f, p.inv_n, p.ph, va, vb);
            const float sz = __ldg(gt.sf[comp][2] + k), cz = __ldg(gt.cpf[comp][2] + k);
            const float dzx = dif(sz, sx, cz, cx);
            const float aa = symbol(sya, cya, dxya, sz, cz, dzx), ab = symbol(syb, cyb, dxyb, sz, cz, dzx);
            // a fast reciprocal (about 2 ulp): the Green step is the fixed point's
            // preconditioner, its operator test bar is 2e-6 of the field
            va = (aa <= thr) ? 0.f : __fdividef(va, aa);
            vb = (ab <= thr) ? 0.f : __fdividef(vb, ab);
            wplace<TY, true>(qr, qi, k, va, vb, n);
          }
        }
        if (k1 == 0) wholes<TY, true>(qr, qi, n);
      }
      wfft<R, quarter ? 1 : -1, false, NK>(sr, si, p.tw1, p.ph, lane, X);
      if (lane < Q) {
#pragma unroll
        for (int k2 = 0; k2 < NK; ++k2) {
          const int k = k1 + R * k2;
          if (k < len) {
            float va, vb;
            wpost<TY, true>(X[k2], k, n, p.sc, p.inv_n, p.ph, va, vb);
            tile[k * RPCP + ra] = va;
            tile[k * RPCP + ra + 1] = vb;
          }
        }
      }
    }
  }
  __syncthreads();
  const long long ob = (long long)comp * p.NN + (long long)kx * p.out_outer + row0;
  for (int e = threadIdx.x; e < len * RPC; e += NW * 32) {
    const int k = e / RPC, r = e - k * RPC;
    if (r < nvalid) p.out[ob + (long long)k * p.out_k + r] = tile[k * RPCP + r];
  }
}

namespace {

constexpr int WNW = 4;   // warps per CTA

// per-warp scratch, then the CTA's tile: len x (RPC + 1) (transposed output) or
// RPC x (len | 1) (row output)
template <int R>
size_t wfft_smem(int len, bool transposed) {
  constexpr int RPC = 2 * WPlan<R>::P * WNW;
  const size_t tile = transposed ? (size_t)len * (RPC + 1) : (size_t)RPC * (size_t)(len | 1);
  return (size_t)WNW * 2 * WPlan<R>::SW * sizeof(float) + tile * sizeof(float);
}

template <typename K>
int wfft_attr(K kernel, size_t sm, size_t& done) {
  if (sm <= done) return 0;
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return (int)e;
  done = sm;
  return 0;
}

// Rows per CTA: the fewest CTAs of at most RPC rows, the rows spread evenly over them (an
// even count, so that row pairs never straddle two CTAs); the n + 1 rows of a
// non-periodic axis would otherwise leave a last CTA with a single row.
template <int R>
int balanced_rows(int nrows) {
  constexpr int RPC = 2 * WPlan<R>::P * WNW;
  const int tiles = (nrows + RPC - 1) / RPC;
  int rpt = (nrows + tiles - 1) / tiles;
  rpt += rpt & 1;
  return rpt < RPC ? rpt : RPC;
}

template <int R, int MODE, int TY, bool INV>
int launch_pass_k(const WfftPass& q, dim3 grd, cudaStream_t s, const Ctrl* ctrl) {
  const size_t sm = wfft_smem<R>(q.len, MODE == 0);
  static size_t attr = 48 * 1024;
  if (int e = wfft_attr(k_wfft<R, WNW, MODE, TY, INV>, sm, attr)) return e;
  k_wfft<R, WNW, MODE, TY, INV><<<grd, WNW * 32, sm, s>>>(q, ctrl);
  return (int)cudaGetLastError();
}
template <int R, int MODE, bool INV>
int launch_pass_ty(int ty, const WfftPass& q, dim3 grd, cudaStream_t s, const Ctrl* ctrl) {
  switch (ty) {
    case T_DCT1: return launch_pass_k<R, MODE, T_DCT1, INV>(q, grd, s, ctrl);
    case T_DCT3: return launch_pass_k<R, MODE, T_DCT3, INV>(q, grd, s, ctrl);
    case T_DST1: return launch_pass_k<R, MODE, T_DST1, INV>(q, grd, s, ctrl);
    default: return launch_pass_k<R, MODE, T_DST3, INV>(q, grd, s, ctrl);
  }
}
template <int R>
int launch_pass_R(const WfftPass& p0, int mode, int nouter, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  WfftPass p = p0;
  p.rpt = balanced_rows<R>(p.nrows);
  dim3 grd((unsigned)((p.nrows + p.rpt - 1) / p.rpt), (unsigned)nouter, 1u);
  // one launch per run of consecutive components of equal type
  for (int c = 0; c < ncomp;) {
    const int ty = p0.type[p0.comp0 + c];
    int m = 1;
    while (c + m < ncomp && p0.type[p0.comp0 + c + m] == ty) ++m;
    WfftPass q = p;
    q.comp0 = p0.comp0 + c;
    grd.z = (unsigned)m;
    int e;
    if (mode == 0) e = p.inverse ? launch_pass_ty<R, 0, true>(ty, q, grd, s, ctrl) : launch_pass_ty<R, 0, false>(ty, q, grd, s, ctrl);
    else e = p.inverse ? launch_pass_ty<R, 2, true>(ty, q, grd, s, ctrl) : launch_pass_ty<R, 2, false>(ty, q, grd, s, ctrl);
    if (e) return e;
    c += m;
  }
  return 0;
}

template <int R>
int launch_zg_R(const WfftPass& p0, const GreenTables& gt, float l0, float m2, float ih2, int scheme, int nouter,
                int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  WfftPass p = p0;
  p.rpt = balanced_rows<R>(p.nrows);
  dim3 grd((unsigned)((p.nrows + p.rpt - 1) / p.rpt), (unsigned)nouter, (unsigned)ncomp);
  const size_t sm = wfft_smem<R>(p.len, true);
  // one launch per run of consecutive components of equal type
  for (int c = 0; c < ncomp;) {
    const int ty = p0.type[p0.comp0 + c];
    int m = 1;
    while (c + m < ncomp && p0.type[p0.comp0 + c + m] == ty) ++m;
    WfftPass q = p;
    q.comp0 = p0.comp0 + c;
    grd.z = (unsigned)m;
    int e = 0;
    auto go = [&](auto kern, size_t& attr) {
      if ((e = wfft_attr(kern, sm, attr))) return;
      kern<<<grd, WNW * 32, sm, s>>>(q, gt, l0, m2, ih2, scheme, ctrl);
      e = (int)cudaGetLastError();
    };
    static size_t attr[4] = {48 * 1024, 48 * 1024, 48 * 1024, 48 * 1024};
    switch (ty) {
      case T_DCT1: go(k_wfft_zg<R, WNW, T_DCT1>, attr[0]); break;
      case T_DCT3: go(k_wfft_zg<R, WNW, T_DCT3>, attr[1]); break;
      case T_DST1: go(k_wfft_zg<R, WNW, T_DST1>, attr[2]); break;
      default: go(k_wfft_zg<R, WNW, T_DST3>, attr[3]); break;
    }
    if (e) return e;
    c += m;
  }
  return 0;
}

int launch_pass(int R, const WfftPass& p, int mode, int nouter, int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  switch (R) {
    case 2: return launch_pass_R<2>(p, mode, nouter, ncomp, ctrl, s);
    case 3: return launch_pass_R<3>(p, mode, nouter, ncomp, ctrl, s);
    case 4: return launch_pass_R<4>(p, mode, nouter, ncomp, ctrl, s);
    case 6: return launch_pass_R<6>(p, mode, nouter, ncomp, ctrl, s);
    case 8: return launch_pass_R<8>(p, mode, nouter, ncomp, ctrl, s);
    case 12: return launch_pass_R<12>(p, mode, nouter, ncomp, ctrl, s);
    case 16: return launch_pass_R<16>(p, mode, nouter, ncomp, ctrl, s);
    case 24: return launch_pass_R<24>(p, mode, nouter, ncomp, ctrl, s);
    case 32: return launch_pass_R<32>(p, mode, nouter, ncomp, ctrl, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

int launch_zg(int R, const WfftPass& p, const GreenTables& gt, float l0, float m2, float ih2, int scheme, int nouter,
              int ncomp, const Ctrl* ctrl, cudaStream_t s) {
  switch (R) {
    case 2: return launch_zg_R<2>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 3: return launch_zg_R<3>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 4: return launch_zg_R<4>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 6: return launch_zg_R<6>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 8: return launch_zg_R<8>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 12: return launch_zg_R<12>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 16: return launch_zg_R<16>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 24: return launch_zg_R<24>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    case 32: return launch_zg_R<32>(p, gt, l0, m2, ih2, scheme, nouter, ncomp, ctrl, s);
    default: return (int)cudaErrorInvalidValue;
  }
}

}  // namespace

int wfft_radix(int L) {
  if (L % 32 != 0) return 0;
  const int R = L / 32;
  switch (R) {
    case 2: case 3: case 4: case 6: case 8: case 12: case 16: case 24: case 32: return R;
    default: return 0;
  }
}

bool wfft_supported(const GridDev& g, const TransformTables& tt) {
  if (g.ref_iso) return false;
  for (int d = 0; d < 3; ++d) {
    if (g.periodic[d] || !tt.fft[d].use || !tt.fft[d].tw1) return false;
    if (tt.fft[d].L != 2 * g.nvox[d] || !wfft_radix(tt.fft[d].L)) return false;
  }
  return true;
}

// The five sweeps of the Green step (see the table at the top of this file).  b1 / b2:
// two work fields of 3 x nnodes floats; the input (or ring slot) is read by the first
// sweep only; with incr the last sweep adds its result to u~ and stores it as the step,
// otherwise it writes `out` (which may be b2: the last sweep reads each row before
// writing it).
int launch_wfft_green(const GridDev& g, const TransformTables& tt, const float* in, void* const* in_ring, float* b1,
                      float* b2, float* out, const IncrTarget* incr, int comp0, int ncomp, const Ctrl* ctrl,
                      cudaStream_t s, void (*mark)(int, cudaStream_t)) {
  const long long nx = g.nn[0], ny = g.nn[1], nz = g.nn[2];
  auto base = [&](int axis, int inverse) {
    WfftPass p{};
    p.len = g.nn[axis];
    p.n = g.nvox[axis];
    p.NN = g.nnodes;
    for (int c = 0; c < 3; ++c) p.type[c] = tt.types[c][axis];
    p.inverse = inverse;
    p.sc = inverse ? (float)(2.0 / g.nvox[axis]) : 1.f;
    p.inv_n = (float)(1.0 / g.nvox[axis]);
    p.tw1 = (const float2*)tt.fft[axis].tw1;
    p.ph = (const float2*)tt.fft[axis].ph;
    p.comp0 = comp0;
    return p;
  };
  // fx: natural -> T1 [c][z][kx][y]
  WfftPass p = base(0, 0);
  p.in = in;
  p.in_ring = in_ring;
  p.out = b1;
  p.nrows = (int)ny;
  p.in_outer = nx * ny;
  p.in_row = nx;
  p.out_outer = nx * ny;
  p.out_k = ny;
  if (int e = launch_pass(wfft_radix(tt.fft[0].L), p, 0, (int)nz, ncomp, ctrl, s)) return e;
  // fy: T1 -> T2 [c][kx][ky][z]
  p = base(1, 0);
  p.in = b1;
  p.out = b2;
  p.nrows = (int)nz;
  p.in_outer = ny;
  p.in_row = nx * ny;
  p.out_outer = ny * nz;
  p.out_k = nz;
  if (int e = launch_pass(wfft_radix(tt.fft[1].L), p, 0, (int)nx, ncomp, ctrl, s)) return e;
  if (mark) mark(4, s);
  // zg: T2 -> T3 [c][z][kx][ky]
  p = base(2, 1);
  p.in = b2;
  p.out = b1;
  p.nrows = (int)ny;
  p.in_outer = ny * nz;
  p.in_row = nz;
  p.out_outer = ny;
  p.out_k = nx * ny;
  GreenTables gt;
  for (int c = 0; c < 3; ++c) {
    for (int d = 0; d < 3; ++d) {
      gt.s[c][d] = tt.sin2q[c][d];
      gt.cp[c][d] = tt.cos2q[c][d];
      gt.sf[c][d] = tt.sin2q_f[c][d];
      gt.cpf[c][d] = tt.cos2q_f[c][d];
    }
    gt.null_thr[c] = tt.null_thr[c];
    gt.null_thr_f[c] = (float)tt.null_thr[c];
  }
  const float l0 = (float)tt.lam0, m2 = (float)(2.0 * tt.mu0), ih2 = (float)(4.0 / (g.h * g.h));
  if (int e = launch_zg(wfft_radix(tt.fft[2].L), p, gt, l0, m2, ih2, g.scheme, (int)nx, ncomp, ctrl, s)) return e;
  if (mark) mark(5, s);
  // iy: T3 -> T4 [c][z][y][kx]
  p = base(1, 1);
  p.in = b1;
  p.out = b2;
  p.nrows = (int)nx;
  p.in_outer = nx * ny;
  p.in_row = ny;
  p.out_outer = nx * ny;
  p.out_k = nx;
  if (int e = launch_pass(wfft_radix(tt.fft[1].L), p, 0, (int)nz, ncomp, ctrl, s)) return e;
  // ix: T4 -> natural rows (or the increment)
  p = base(0, 1);
  p.in = b2;
  p.out = out;
  p.nrows = (int)ny;
  p.in_outer = nx * ny;
  p.in_row = nx;
  if (incr) {
    p.uhi = incr->uhi;
    p.ulo = incr->ulo;
    p.step = (float*)incr->step;
  }
  const int e = launch_pass(wfft_radix(tt.fft[0].L), p, 2, (int)nz, ncomp, ctrl, s);
  if (mark) mark(6, s);
  return e;
}

}  // namespace dtt
