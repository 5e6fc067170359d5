// lise_fft.cuh -- shared-memory line FFTs for the spectral Laplacian.
//
// The kinetic operator of the TDSLDA Hamiltonian is -(alpha/2) lap applied as
// D^(2) f = F^-1[(ik)^2 F f] with an unnormalised forward transform and a 1/N
// inverse (arXiv:2009.00745, Sec. "Discretization").  Lines of length
// N = N1 * N2 held in shared memory are transformed by the four-step scheme:
//   phase 1: for each j2 < N2, an N1-point DFT over j1 of x[j2 + N2 j1], then
//            the twiddle exp(S 2 pi i j2 k1 / N), written back in place;
//   phase 2: for each k1 < N1, an N2-point DFT over j2 of the phase-1 output at
//            j2 + N2 k1, giving X[k1 + N1 k2] (natural order).
// S = -1 is the forward transform, S = +1 the (unnormalised) inverse.  All
// threads of the block cooperate; a line's work items are spread so that
// consecutive threads handle consecutive lines.
#pragma once
#include <cuda_runtime.h>

namespace lise {

template <typename R> struct Cx;
template <> struct Cx<double> { using T = double2; };
template <> struct Cx<float> { using T = float2; };

template <typename T> __device__ __forceinline__ T cadd(T a, T b) { return T{a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { return T{a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  return T{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ T cconj(T a) { return T{a.x, -a.y}; }
template <typename T, typename R> __device__ __forceinline__ T cscale(T a, R s) { return T{a.x * s, a.y * s}; }
// multiply by i*S
template <int S, typename T> __device__ __forceinline__ T mul_iS(T a) {
  return S > 0 ? T{-a.y, a.x} : T{a.y, -a.x};
}
// multiply by exp(S i pi/4) = (1 + S i)/sqrt(2) and exp(S 3 i pi/4) = (-1 + S i)/sqrt(2)
template <int S, typename T, typename R> __device__ __forceinline__ T mul_w8_1(T a, R r2) {
  // (x + iy)(1 + S i) = (x - S y) + i(y + S x)
  return S > 0 ? T{(a.x - a.y) * r2, (a.y + a.x) * r2} : T{(a.x + a.y) * r2, (a.y - a.x) * r2};
}
template <int S, typename T, typename R> __device__ __forceinline__ T mul_w8_3(T a, R r2) {
  // (x + iy)(-1 + S i) = (-x - S y) + i(-y + S x)
  return S > 0 ? T{(-a.x - a.y) * r2, (a.x - a.y) * r2} : T{(a.y - a.x) * r2, (-a.y - a.x) * r2};
}

// Mathematical constants of the small DFTs (cos and sin of 2 pi k / R).
template <typename R> struct K {
  static constexpr R r2 = R(0.70710678118654752440084436210485);   // 1/sqrt(2)
  static constexpr R s3 = R(0.86602540378443864676372317075294);   // sin(2 pi/3)
  static constexpr R c51 = R(0.30901699437494742410229341718282);  // cos(2 pi/5)
  static constexpr R c52 = R(-0.80901699437494742410229341718282); // cos(4 pi/5)
  static constexpr R s51 = R(0.95105651629515357211643933337938);  // sin(2 pi/5)
  static constexpr R s52 = R(0.58778525229247312916870595463907);  // sin(4 pi/5)
};

// In-register DFT of size R: x_k <- sum_j x_j exp(S 2 pi i j k / R).
template <int N, int S, typename R> struct Dft;

template <int S, typename R> struct Dft<1, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T*) {}
};

template <int S, typename R> struct Dft<2, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T* x) {
    T a = x[0], b = x[1];
    x[0] = cadd(a, b);
    x[1] = csub(a, b);
  }
};

template <int S, typename R> struct Dft<3, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T* x) {
    T t1 = cadd(x[1], x[2]);
    T t2 = T{x[0].x - R(0.5) * t1.x, x[0].y - R(0.5) * t1.y};
    T t3 = mul_iS<S>(cscale(csub(x[1], x[2]), K<R>::s3));
    x[0] = cadd(x[0], t1);
    x[1] = cadd(t2, t3);
    x[2] = csub(t2, t3);
  }
};

template <int S, typename R> struct Dft<4, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T* x) {
    T e0 = cadd(x[0], x[2]), e1 = csub(x[0], x[2]);
    T o0 = cadd(x[1], x[3]), o1 = mul_iS<S>(csub(x[1], x[3]));
    x[0] = cadd(e0, o0);
    x[2] = csub(e0, o0);
    x[1] = cadd(e1, o1);
    x[3] = csub(e1, o1);
  }
};

template <int S, typename R> struct Dft<5, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T* x) {
    T a1 = cadd(x[1], x[4]), b1 = csub(x[1], x[4]);
    T a2 = cadd(x[2], x[3]), b2 = csub(x[2], x[3]);
    T x0 = x[0];
    T r1 = T{x0.x + K<R>::c51 * a1.x + K<R>::c52 * a2.x, x0.y + K<R>::c51 * a1.y + K<R>::c52 * a2.y};
    T r2 = T{x0.x + K<R>::c52 * a1.x + K<R>::c51 * a2.x, x0.y + K<R>::c52 * a1.y + K<R>::c51 * a2.y};
    T i1 = mul_iS<S>(T{K<R>::s51 * b1.x + K<R>::s52 * b2.x, K<R>::s51 * b1.y + K<R>::s52 * b2.y});
    T i2 = mul_iS<S>(T{K<R>::s52 * b1.x - K<R>::s51 * b2.x, K<R>::s52 * b1.y - K<R>::s51 * b2.y});
    x[0] = cadd(x0, cadd(a1, a2));
    x[1] = cadd(r1, i1);
    x[4] = csub(r1, i1);
    x[2] = cadd(r2, i2);
    x[3] = csub(r2, i2);
  }
};

template <int S, typename R> struct Dft<6, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T* x) {
    // even/odd split into two 3-point DFTs; w6 = exp(S i pi/3) = 1/2 + S i sqrt(3)/2
    T e[3] = {x[0], x[2], x[4]};
    T o[3] = {x[1], x[3], x[5]};
    Dft<3, S, R>::run(e);
    Dft<3, S, R>::run(o);
    T o1 = T{R(0.5) * o[1].x, R(0.5) * o[1].y};
    o1 = cadd(o1, mul_iS<S>(cscale(o[1], K<R>::s3)));             // w6 * o1
    T o2 = T{R(-0.5) * o[2].x, R(-0.5) * o[2].y};
    o2 = cadd(o2, mul_iS<S>(cscale(o[2], K<R>::s3)));             // w6^2 * o2
    x[0] = cadd(e[0], o[0]);
    x[3] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[4] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[5] = csub(e[2], o2);
  }
};

template <int S, typename R> struct Dft<8, S, R> {
  using T = typename Cx<R>::T;
  static __device__ __forceinline__ void run(T* x) {
    T e[4] = {x[0], x[2], x[4], x[6]};
    T o[4] = {x[1], x[3], x[5], x[7]};
    Dft<4, S, R>::run(e);
    Dft<4, S, R>::run(o);
    T o1 = mul_w8_1<S>(o[1], K<R>::r2);
    T o2 = mul_iS<S>(o[2]);
    T o3 = mul_w8_3<S>(o[3], K<R>::r2);
    x[0] = cadd(e[0], o[0]);
    x[4] = csub(e[0], o[0]);
    x[1] = cadd(e[1], o1);
    x[5] = csub(e[1], o1);
    x[2] = cadd(e[2], o2);
    x[6] = csub(e[2], o2);
    x[3] = cadd(e[3], o3);
    x[7] = csub(e[3], o3);
  }
};

// Factorisation N = N1 * N2 used for each supported line length.
template <int N> struct Plan;
template <> struct Plan<8> { static constexpr int N1 = 2, N2 = 4; };
template <> struct Plan<12> { static constexpr int N1 = 4, N2 = 3; };
template <> struct Plan<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Plan<20> { static constexpr int N1 = 4, N2 = 5; };
template <> struct Plan<24> { static constexpr int N1 = 4, N2 = 6; };
template <> struct Plan<32> { static constexpr int N1 = 4, N2 = 8; };
template <> struct Plan<40> { static constexpr int N1 = 8, N2 = 5; };
template <> struct Plan<48> { static constexpr int N1 = 8, N2 = 6; };
template <> struct Plan<64> { static constexpr int N1 = 8, N2 = 8; };

// Phase 1 of the four-step transform on NL lines with NT threads.  base(l)
// gives the shared-memory offset (in elements) of line l, es the element
// stride.  tw[j2 * N1 + k1] = exp(-2 pi i j2 k1 / N) (forward twiddles; the
// inverse uses their conjugates).
template <int N, int S, typename R, int NL, int NT, typename Base>
__device__ __forceinline__ void fft_phase1(typename Cx<R>::T* buf, Base base, int es,
                                           const typename Cx<R>::T* tw) {
  using T = typename Cx<R>::T;
  constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
  constexpr int TOTAL = NL * N2;
  constexpr int ITEMS = (TOTAL + NT - 1) / NT;
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    int it = threadIdx.x + r * NT;
    if (TOTAL % NT == 0 || it < TOTAL) {
      int l = it % NL, j2 = it / NL;
      T* p = buf + base(l) + j2 * es;
      T a[N1];
#pragma unroll
      for (int j1 = 0; j1 < N1; ++j1) a[j1] = p[j1 * N2 * es];
      Dft<N1, S, R>::run(a);
      if (j2 != 0) {  // the j2 = 0 twiddles are 1 (warp-uniform: lines are the fast index)
#pragma unroll
        for (int k1 = 1; k1 < N1; ++k1) {
          T w = tw[j2 * N1 + k1];
          if (S > 0) w.y = -w.y;
          a[k1] = cmul(a[k1], w);
        }
      }
#pragma unroll
      for (int k1 = 0; k1 < N1; ++k1) p[k1 * N2 * es] = a[k1];
    }
  }
}

// Phase 2; post(l, k, value) may transform each output element X[k] of line l
// (e.g. multiply by the kinetic factor) before it is stored.  Contains the
// block-wide barrier that separates the in-place loads from the stores.
template <int N, int S, typename R, int NL, int NT, typename Base, typename Post>
__device__ __forceinline__ void fft_phase2(typename Cx<R>::T* buf, Base base, int es, Post post) {
  using T = typename Cx<R>::T;
  constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
  constexpr int TOTAL = NL * N1;
  constexpr int ITEMS = (TOTAL + NT - 1) / NT;
  T b[ITEMS][N2];
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    int it = threadIdx.x + r * NT;
    if (TOTAL % NT == 0 || it < TOTAL) {
      int l = it % NL, k1 = it / NL;
      T* p = buf + base(l) + k1 * N2 * es;
#pragma unroll
      for (int j2 = 0; j2 < N2; ++j2) b[r][j2] = p[j2 * es];
      Dft<N2, S, R>::run(b[r]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < ITEMS; ++r) {
    int it = threadIdx.x + r * NT;
    if (TOTAL % NT == 0 || it < TOTAL) {
      int l = it % NL, k1 = it / NL;
      T* p = buf + base(l);
#pragma unroll
      for (int k2 = 0; k2 < N2; ++k2) {
        int k = k1 + N1 * k2;
        p[k * es] = post(l, k, b[r][k2]);
      }
    }
  }
}

struct Identity {
  template <typename T> __device__ __forceinline__ T operator()(int, int, T v) const { return v; }
  template <typename T> __device__ __forceinline__ T operator()(int, T v) const { return v; }
};

// The same four-step transform of one line held by one thread in registers (x in natural
// order in and out; post(k, value) as in fft_phase2): the same butterflies, twiddles and
// operation order as fft_phase1 and fft_phase2, so the values are those of the
// shared-memory version.  Every index is a compile-time constant (fully unrolled).
template <int N, int S, typename R, typename Post>
__device__ __forceinline__ void line_fft(typename Cx<R>::T (&x)[N], const typename Cx<R>::T* tw, Post post) {
  using T = typename Cx<R>::T;
  constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2;
#pragma unroll
  for (int j2 = 0; j2 < N2; ++j2) {
    T a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) a[j1] = x[j2 + N2 * j1];
    Dft<N1, S, R>::run(a);
    if (j2 != 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) {
        T w = tw[j2 * N1 + k1];
        if (S > 0) w.y = -w.y;
        a[k1] = cmul(a[k1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) x[j2 + N2 * k1] = a[k1];
  }
  T y[N];
#pragma unroll
  for (int k1 = 0; k1 < N1; ++k1) {
    T b[N2];
#pragma unroll
    for (int j2 = 0; j2 < N2; ++j2) b[j2] = x[k1 * N2 + j2];
    Dft<N2, S, R>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) y[k1 + N1 * k2] = post(k1 + N1 * k2, b[k2]);
  }
#pragma unroll
  for (int k = 0; k < N; ++k) x[k] = y[k];
}

// Full line transform (both phases), with barriers after each phase.
template <int N, int S, typename R, int NL, int NT, typename Base, typename Post>
__device__ __forceinline__ void fft_lines(typename Cx<R>::T* buf, Base base, int es,
                                          const typename Cx<R>::T* tw, Post post) {
  fft_phase1<N, S, R, NL, NT>(buf, base, es, tw);
  __syncthreads();
  fft_phase2<N, S, R, NL, NT>(buf, base, es, post);
  __syncthreads();
}

// The same transform of one line shared by two threads (N1 and N2 even): thread s holds the
// line positions p = 2 m + s in L[m], m < N/2, on input and on output.  Phase 1: the thread's
// N1-point DFTs are those of j2 = 2 jj + s; phase 2 needs, for k1 = 2 kk + s, the phase-1
// values of every j2: the ones of the other parity come from the partner thread (lane ^ 16,
// one shuffle per real word).  The butterflies, twiddles and operation order are those of
// fft_phase1 and fft_phase2 (the shuffles and selects only move values), so the values are
// those of the shared-memory version.  Every register index is a compile-time constant.
template <int N, int S, typename Post>
__device__ __forceinline__ void half_line_fft(float2 (&L)[N / 2], const float2* tw, int s, Post post) {
  constexpr int N1 = Plan<N>::N1, N2 = Plan<N>::N2, H1 = N1 / 2, H2 = N2 / 2;
  static_assert(N1 % 2 == 0 && N2 % 2 == 0, "half lines need even factors");
  float2 P[H2][N1];  // phase-1 output of j2 = 2 jj + s at k1
#pragma unroll
  for (int jj = 0; jj < H2; ++jj) {
    const int j2 = 2 * jj + s;
    float2 a[N1];
#pragma unroll
    for (int j1 = 0; j1 < N1; ++j1) a[j1] = L[jj + H2 * j1];  // position j2 + N2 j1
    Dft<N1, S, float>::run(a);
    if (j2 != 0) {
#pragma unroll
      for (int k1 = 1; k1 < N1; ++k1) {
        float2 w = tw[j2 * N1 + k1];
        if (S > 0) w.y = -w.y;
        a[k1] = cmul(a[k1], w);
      }
    }
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) P[jj][k1] = a[k1];
  }
#pragma unroll
  for (int kk = 0; kk < H1; ++kk) {
    // k1 = 2 kk + s: own values at j2 = 2 jj + s, the partner's at j2 = 2 jj + 1 - s
    float2 b[N2];
#pragma unroll
    for (int jj = 0; jj < H2; ++jj) {
      const float2 keep = s ? P[jj][2 * kk + 1] : P[jj][2 * kk];
      const float2 send = s ? P[jj][2 * kk] : P[jj][2 * kk + 1];
      float2 recv;
      recv.x = __shfl_xor_sync(0xFFFFFFFFu, send.x, 16);
      recv.y = __shfl_xor_sync(0xFFFFFFFFu, send.y, 16);
      b[2 * jj] = s ? recv : keep;
      b[2 * jj + 1] = s ? keep : recv;
    }
    Dft<N2, S, float>::run(b);
#pragma unroll
    for (int k2 = 0; k2 < N2; ++k2) L[kk + H1 * k2] = post(2 * kk + s + N1 * k2, b[k2]);  // position k1 + N1 k2
  }
}

}  // namespace lise
