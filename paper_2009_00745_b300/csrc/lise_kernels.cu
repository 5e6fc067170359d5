// lise_kernels.cu -- device kernels of the two-component TDSLDA step and their
// launchers.  See lise_kernels.cuh for the operator split and the modes.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "lise_kernels.cuh"
#include "lise_ozaki.cuh"
#include "lise_umma.cuh"

namespace lise {

// binary64 <-> binary32 conversions done with integer operations on the bit
// patterns (IEEE 754 layouts), so that they do not occupy the FP64 pipe, which
// on this GPU runs at 1/64 of the FP32 rate and also executes F2F.
// Round to nearest even; results below the binary32 normal range flush to a
// signed zero (the path's values are many orders of magnitude above it).
__device__ __forceinline__ float d2f_bits(double x) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7FFu);
  const unsigned m = ((hi & 0xFFFFFu) << 3) | (lo >> 29);   // top 23 fraction bits
  const unsigned rest = lo & 0x1FFFFFFFu;                     // 29 bits below them
  const int fe = e - 896;                                     // rebias 1023 -> 127
  unsigned r = ((unsigned)fe << 23) + m;
  r += (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;  // carries into the exponent
  if (fe <= 0) r = 0u;
  if (fe >= 255) r = (e == 0x7FF && ((hi & 0xFFFFFu) | lo)) ? 0x7FC00000u : 0x7F800000u;
  return __uint_as_float(sign | r);
}
__device__ __forceinline__ double f2d_bits(float f) {
  const unsigned b = __float_as_uint(f);
  const unsigned sign = b & 0x80000000u;
  const unsigned e = (b >> 23) & 0xFFu;
  const unsigned m = b & 0x7FFFFFu;
  unsigned hi, lo;
  if (e == 0u) {  // zero (binary32 subnormals flush to zero)
    hi = sign;
    lo = 0u;
  } else if (e == 0xFFu) {
    hi = sign | 0x7FF00000u | (m >> 3) | (m ? 0x80000u : 0u);
    lo = m << 29;
  } else {
    hi = sign | ((e + 896u) << 20) | (m >> 3);
    lo = m << 29;
  }
  return __hiloint2double((int)hi, (int)lo);
}

template <typename R> __device__ __forceinline__ typename Cx<R>::T to_r(double2 v);
template <> __device__ __forceinline__ double2 to_r<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_r<float>(double2 v) {
  return make_float2(d2f_bits(v.x), d2f_bits(v.y));
}
// Conversion on the hardware path (F2F, executed by the FP64 pipe): used where that
// pipe is otherwise idle (the planes kernel), to spare the integer pipe.
template <typename R> __device__ __forceinline__ typename Cx<R>::T to_r_hw(double2 v);
template <> __device__ __forceinline__ double2 to_r_hw<double>(double2 v) { return v; }
template <> __device__ __forceinline__ float2 to_r_hw<float>(double2 v) {
  return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}
__device__ __forceinline__ double2 to_d(double2 v) { return v; }
__device__ __forceinline__ double2 to_d(float2 v) { return make_double2(f2d_bits(v.x), f2d_bits(v.y)); }

// fused multiply-add in the operands' own precision
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }

__device__ __forceinline__ double2 dadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 dsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 dscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ double2 dmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// The predictor's derivative sums of the FP64 path, evaluated exactly in integers:
//   sp = 119 f - 99 e0 + 69 e1 - 17 e2   (pt = h/48 sp, Eq. p)
//   sr =  68 f - 102 e0 + 68 e1 - 17 e2  (pt - ct = h/48 sr, with ct of Eq. c)
// The four significands are aligned to the largest exponent (bits below 2^-52 of the
// largest value are dropped), the sums are exact in 64-bit integers (|sum| < 2^62) and
// each is rounded once to FP64 by integer operations (to nearest even, as the FP64 unit's
// conversion would; on the integer pipe, which has more room in this FP64-bound launch: 0.9%
// faster than converting sr on the FP64 unit).
// Non-finite or extreme inputs take the FP64 formula (which keeps NaN and inf).
__device__ __forceinline__ void pred_sums(double f, double e0, double e1, double e2, double& sp, double& sr) {
  const double v[4] = {f, e0, e1, e2};
  unsigned long long b[4];
  int ex[4], emax = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    b[k] = (unsigned long long)__double_as_longlong(v[k]);
    ex[k] = (int)((b[k] >> 52) & 0x7FF);
    emax = max(emax, ex[k]);
  }
  if (emax == 0 || emax > 2000) {
    sp = 119.0 * f - 99.0 * e0 + 69.0 * e1 - 17.0 * e2;
    sr = 68.0 * f - 102.0 * e0 + 68.0 * e1 - 17.0 * e2;
    return;
  }
  long long A[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    unsigned long long m = ex[k] ? ((b[k] & 0xFFFFFFFFFFFFFull) | (1ull << 52)) : 0ull;
    const int sh = emax - ex[k];
    m = sh < 64 ? (m >> sh) : 0ull;
    A[k] = (b[k] >> 63) ? -(long long)m : (long long)m;
  }
  const int sc = emax - 1075;  // a significand aligned to emax is worth 2^(emax - 1075)
  sp = oz::to_double(119 * A[0] - 99 * A[1] + 69 * A[2] - 17 * A[3], sc);
  sr = oz::to_double(68 * A[0] - 102 * A[1] + 68 * A[2] - 17 * A[3], sc);
}

// v / 2 through an exponent decrement on the integer pipe: exact for normal v above the
// smallest normal exponent; zero, subnormals and the smallest normal binade are returned
// unchanged (an absolute difference below 2^-1022), infinities and NaN as they are.
__device__ __forceinline__ double half_exp(double v) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7FF);
  return (e > 1 && e < 0x7FF) ? __longlong_as_double(b - (1ll << 52)) : v;
}

// sn += |v|^2 ; nu += u conj(v)  (the factor 2 of n = 2 sum |v|^2 is applied where the
// partial sums are stored; scaling by 2 is exact, so the order does not matter)
__device__ __forceinline__ void dens_acc(double2 u, double2 v, double& sn, double& sr, double& si) {
  sn = fma(v.x, v.x, fma(v.y, v.y, sn));
  sr = fma(u.x, v.x, fma(u.y, v.y, sr));
  si = fma(u.y, v.x, fma(-u.x, v.y, si));
}
// The same from FP32 operands (the mixed path, whose densities only set the potentials
// of its FP32 H psi): products in FP32 (relative rounding 2^-24, the level of the FP32
// potentials themselves), compensated (Kahan) FP32 sums over the thread's states (error
// a few units of 2^-24 of the sum, independent of the count), folded into the FP64
// partial sums at the end; the sum over groups is FP64 (Neumaier, k_reduce).
struct KahanF {
  float s = 0.f, c = 0.f;  // sum and the negative of its lost low part
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return f2d_bits(s) - f2d_bits(c); }
};
struct DensF {
  KahanF n, r, i;
};
__device__ __forceinline__ void dens_acc(float2 u, float2 v, DensF& d) {
  d.n.add(fmaf(v.x, v.x, v.y * v.y));
  d.r.add(fmaf(u.x, v.x, u.y * v.y));
  d.i.add(fmaf(u.y, v.x, -(u.x * v.y)));
}
__device__ __forceinline__ void dens_fold(const DensF& d, double& sn, double& sr, double& si) {
  sn += d.n.value();
  sr += d.r.value();
  si += d.i.value();
}


// Padded-plane tile count per block for the planes kernel.
template <int N> struct PlanesPB { static constexpr int v = N <= 8 ? 8 : (N <= 16 ? 4 : (N <= 32 ? 2 : 1)); };

// ------------------------------------------------------------------ planes --
// The kinetic factor's multiply, rounded on its own (never fused with the additions of the
// transform that follows: in the register-line kernel the product stays in registers, and the
// two planes kernels must round identically).
__device__ __forceinline__ float2 kin_mul(float2 v, float f) { return make_float2(__fmul_rn(v.x, f), __fmul_rn(v.y, f)); }
__device__ __forceinline__ double2 kin_mul(double2 v, double f) { return make_double2(__dmul_rn(v.x, f), __dmul_rn(v.y, f)); }

// The block's PB planes of the operand into shared memory (rows padded to N + 1 elements, so
// that row and column lines are both conflict-free), with the twiddles and kinetic factors;
// returns the number of planes the block holds (NT threads).
template <typename R, int N, int PB, int NT>
__device__ __forceinline__ int planes_load(const PlanesArgs& a, const long block, typename Cx<R>::T* buf,
                                           typename Cx<R>::T* tw, R* hk) {
  using T = typename Cx<R>::T;
  constexpr int NP = N + 1;   // padded row stride (conflict-free row and column lines)
  constexpr int PS = N * NP;  // plane stride
  const T* twg = reinterpret_cast<const T*>(a.tw);
  const R* hg = reinterpret_cast<const R*>(a.hxy);
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = twg[i];
    hk[i] = hg[i];
  }
  const long plane0 = block * PB;
  const long left = a.n_planes - plane0;
  const int np = left < PB ? (int)left : PB;
  const double2* src = a.x + plane0 * N * N;
  const T* srcr = a.xr ? reinterpret_cast<const T*>(a.xr) + plane0 * N * N : nullptr;
  // a compile-time count of elements per thread: all of a thread's loads are issued
  // before the first store (several global loads in flight per thread)
  constexpr int EPT = (PB * N * N + NT - 1) / NT;
  T v[EPT];
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = threadIdx.x + e * NT;
    const int pl = i / (N * N);
    v[e] = T{R(0), R(0)};
    if (i < PB * N * N && pl < np) v[e] = srcr ? srcr[i] : to_r_hw<R>(src[i]);
  }
#pragma unroll
  for (int e = 0; e < EPT; ++e) {
    const int i = threadIdx.x + e * NT;
    const int pl = i / (N * N), r = i % (N * N);
    if (i < PB * N * N) buf[pl * PS + (r / N) * NP + (r % N)] = v[e];
  }
  return np;
}

// The block's np planes of T_xy x from shared memory, coalesced.
template <typename R, int N, int PB, int NT>
__device__ __forceinline__ void planes_store(const PlanesArgs& a, const long block, const int np,
                                            const typename Cx<R>::T* buf) {
  using T = typename Cx<R>::T;
  constexpr int NP = N + 1, PS = N * NP;
  T* dst = reinterpret_cast<T*>(a.txy) + block * PB * N * N;
  for (int i = threadIdx.x; i < np * N * N; i += NT) {
    int pl = i / (N * N), r = i % (N * N);
    dst[i] = buf[pl * PS + (r / N) * NP + (r % N)];
  }
}

template <typename R, int N, int PB, int NT>
__device__ __forceinline__ void planes_body(const PlanesArgs& a, const long block) {
  using T = typename Cx<R>::T;
  constexpr int NP = N + 1;   // padded row stride (conflict-free row and column lines)
  constexpr int PS = N * NP;  // plane stride
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* tw = buf + PB * PS;
  R* hk = reinterpret_cast<R*>(tw + N);
  const int np = planes_load<R, N, PB, NT>(a, block, buf, tw, hk);
  __syncthreads();
  auto rows = [](int l) { return (l / N) * PS + (l % N) * NP; };
  auto cols = [](int l) { return (l / N) * PS + (l % N); };
  fft_lines<N, -1, R, PB * N, NT>(buf, rows, 1, tw, Identity());
  // forward along y; on store multiply by (alpha/2)(kx^2 + ky^2)/N^2 (line l has kx = l % N)
  fft_lines<N, -1, R, PB * N, NT>(buf, cols, NP, tw, [&](int l, int k, T v) { return kin_mul(v, hk[l % N] + hk[k]); });
  fft_lines<N, +1, R, PB * N, NT>(buf, cols, NP, tw, Identity());
  fft_lines<N, +1, R, PB * N, NT>(buf, rows, 1, tw, Identity());
  planes_store<R, N, PB, NT>(a, block, np, buf);
}

// The same transform with whole lines in registers (FP32 compute precision): one thread per
// line (PB N threads), the plane in shared memory only between the row, column and row passes
// (8 shared-memory accesses per element instead of 18: this kernel is bound by shared-memory
// bandwidth).  The line transforms are line_fft, the same operations in the same order as the
// shared-memory passes: the result is bitwise that of planes_body.
template <int N, int PB>
__device__ __forceinline__ void planes_line_body(const PlanesArgs& a, const long block) {
  using R = float;
  using T = float2;
  constexpr int NT = PB * N, NP = N + 1, PS = N * NP;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* tw = buf + PB * PS;
  R* hk = reinterpret_cast<R*>(tw + N);
  const int np = planes_load<R, N, PB, NT>(a, block, buf, tw, hk);
  __syncthreads();
  const int ln = threadIdx.x % N;  // this thread's row y, then column x, of plane threadIdx.x / N
  T* row = buf + (threadIdx.x / N) * PS + ln * NP;
  T* col = buf + (threadIdx.x / N) * PS + ln;
  T x[N];
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = row[i];
  line_fft<N, -1, R>(x, tw, Identity());
#pragma unroll
  for (int i = 0; i < N; ++i) row[i] = x[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = col[i * NP];
  // forward along y, times (alpha/2)(kx^2 + ky^2)/N^2 (kx = ln), then the inverse along y
  line_fft<N, -1, R>(x, tw, [&](int k, T v) { return kin_mul(v, hk[ln] + hk[k]); });
  line_fft<N, +1, R>(x, tw, Identity());
#pragma unroll
  for (int i = 0; i < N; ++i) col[i * NP] = x[i];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = row[i];
  line_fft<N, +1, R>(x, tw, Identity());
#pragma unroll
  for (int i = 0; i < N; ++i) row[i] = x[i];
  __syncthreads();
  planes_store<R, N, PB, NT>(a, block, np, buf);
}

// The same with each line shared by two threads (lattices of 48 and 64 points, whose whole
// lines do not fit in one thread's registers): 2 PB N threads, half_line_fft.  Warp lanes
// 0-15 hold the even positions of 16 lines, lanes 16-31 the odd positions of the same lines
// (conflict-free shared-memory rows and columns).  Bitwise the result of planes_body.
template <int N, int PB>
__device__ __forceinline__ void planes_half_body(const PlanesArgs& a, const long block) {
  using R = float;
  using T = float2;
  constexpr int NT = 2 * PB * N, NP = N + 1, PS = N * NP, H = N / 2;
  static_assert(PB * N % 16 == 0, "whole warps of lines");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);
  T* tw = buf + PB * PS;
  R* hk = reinterpret_cast<R*>(tw + N);
  const int np = planes_load<R, N, PB, NT>(a, block, buf, tw, hk);
  __syncthreads();
  const int lane = threadIdx.x & 31, s = lane >> 4;
  const int line = 16 * (threadIdx.x >> 5) + (lane & 15);  // of the block's PB N lines
  const int ln = line % N;                                  // row y, then column x
  T* row = buf + (line / N) * PS + ln * NP;
  T* col = buf + (line / N) * PS + ln;
  T L[H];
#pragma unroll
  for (int m = 0; m < H; ++m) L[m] = row[2 * m + s];
  half_line_fft<N, -1>(L, tw, s, Identity());
#pragma unroll
  for (int m = 0; m < H; ++m) row[2 * m + s] = L[m];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < H; ++m) L[m] = col[(2 * m + s) * NP];
  half_line_fft<N, -1>(L, tw, s, [&](int k, T v) { return kin_mul(v, hk[ln] + hk[k]); });
  half_line_fft<N, +1>(L, tw, s, Identity());
#pragma unroll
  for (int m = 0; m < H; ++m) col[(2 * m + s) * NP] = L[m];
  __syncthreads();
#pragma unroll
  for (int m = 0; m < H; ++m) L[m] = row[2 * m + s];
  half_line_fft<N, +1>(L, tw, s, Identity());
#pragma unroll
  for (int m = 0; m < H; ++m) row[2 * m + s] = L[m];
  __syncthreads();
  planes_store<R, N, PB, NT>(a, block, np, buf);
}

// The register-line kernels: one thread per line up to 40 points, two from 48 (LineTpl).
template <int N> struct LineTpl { static constexpr int v = N >= 48 ? 2 : 1; };

// resident blocks of the line kernels: a register budget of about 168 per thread for whole
// lines of 40 points (a line of N complex values takes 2N registers), 128 otherwise
template <int N, int NT>
constexpr int line_min_blocks() {
  constexpr int regs = (N >= 40 && LineTpl<N>::v == 1) ? 168 : 128, w = (NT + 31) / 32 * 32;
  return 65536 / (w * regs) < 1 ? 1 : 65536 / (w * regs);
}

template <int N, int PB>
__device__ __forceinline__ void planes_reg_body(const PlanesArgs& a, const long block) {
  if constexpr (LineTpl<N>::v == 2)
    planes_half_body<N, PB>(a, block);
  else
    planes_line_body<N, PB>(a, block);
}

template <int N, int PB>
__global__ void __launch_bounds__(LineTpl<N>::v * PB * N, line_min_blocks<N, LineTpl<N>::v * PB * N>())
    k_planes_line(PlanesArgs a) {
  planes_reg_body<N, PB>(a, blockIdx.x);
}

template <int N, int PB>
__global__ void __launch_bounds__(LineTpl<N>::v * PB * N, line_min_blocks<N, LineTpl<N>::v * PB * N>())
    k_planes_line_batch(const __grid_constant__ PlanesBatch b) {
  int k = 0;
  while (k + 1 < b.n_seg && (long)blockIdx.x >= b.block0[k + 1]) ++k;
  planes_reg_body<N, PB>(b.seg[k], (long)blockIdx.x - b.block0[k]);
}

template <typename R, int N, int PB, int NT>
__global__ void __launch_bounds__(NT) k_planes(PlanesArgs a) {
  planes_body<R, N, PB, NT>(a, blockIdx.x);
}

// Several evolutions' planes in one launch: segment k covers blocks
// [b.block0[k], b.block0[k + 1]) with the arguments b.seg[k] (one evolution's operand).
template <typename R, int N, int PB, int NT>
__global__ void __launch_bounds__(NT) k_planes_batch(const __grid_constant__ PlanesBatch b) {
  int k = 0;
  while (k + 1 < b.n_seg && (long)blockIdx.x >= b.block0[k + 1]) ++k;
  planes_body<R, N, PB, NT>(b.seg[k], (long)blockIdx.x - b.block0[k]);
}

// --------------------------------------------------------- planes, FP64 MMA --
// T_xy x = T_x x + T_y x on PB planes per block with the FP64-accurate tensor-core
// product of lise_ozaki.cuh.  Groups of lines sharing one exponent: (plane, re/im).
//   T_x: Out[y][x] = sum_x' X[y][x'] D2[x][x']   (data rows y, K = x')
//   T_y: Out[y][x] = sum_y' D2[y][y'] X[y'][x]    (data rows x via a transposed load, K = y')
// Both are exact 64-bit integer sums of one scale, added in shared memory, then
// converted to FP64 once.
template <int N> struct OzPlanes {
  static constexpr int PB = N <= 16 ? 4 : 1;
  static constexpr int RS = N + 8;  // padded digit row (bf16): conflict-free ldmatrix rows
  static constexpr int G = PB * 2;  // exponent groups
  static constexpr size_t dig_bytes = (size_t)oz::S * G * N * RS * 2;
  static constexpr size_t smem = dig_bytes + (size_t)G * N * N * 8;
};

template <int N>
__global__ void __launch_bounds__(256) k_planes_oz(PlanesArgs a) {
  using P = OzPlanes<N>;
  constexpr int PB = P::PB, RS = P::RS, G = P::G;
  constexpr int NT = 256, NW = NT / 32;
  constexpr int KS = N / 16, NTILE = N / 8, MT = G * N / 16;
  constexpr int EPT = PB * N * N / NT;  // elements per thread
  static_assert(PB * N * N % NT == 0, "plane block size");
  // x-adjacent element pairs per thread (two digits per 32-bit shared store) where the 2 NT
  // elements of one pass lie in one plane
  constexpr bool kPair = N * N % (2 * NT) == 0;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned short* dig = reinterpret_cast<unsigned short*>(smem_raw);  // [S][G][N][RS]
  long long* acc64 = reinterpret_cast<long long*>(smem_raw + P::dig_bytes);  // [G][N][N]
  __shared__ unsigned ered[NW][G];
  __shared__ unsigned Eg[G];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  const long plane0 = (long)blockIdx.x * PB;
  const long left = a.n_planes - plane0;
  const int np = left < PB ? (int)left : PB;
  // the operand: x, or xr when the operand is stored in the compute precision (here FP64)
  const double2* src = (a.xr ? reinterpret_cast<const double2*>(a.xr) : a.x) + plane0 * N * N;

  // 1. the operand and the largest exponent of each (plane, re/im) group; each thread
  // holds pairs of x-adjacent elements (element i = 2 (tid + r' NT) + e, r = 2 r' + e)
  double2 v[EPT];
  unsigned em[G];
#pragma unroll
  for (int g = 0; g < G; ++g) em[g] = 0;
#pragma unroll
  for (int r = 0; r < EPT; ++r) {
    const int i = kPair ? 2 * (tid + (r >> 1) * NT) + (r & 1) : tid + r * NT;
    const int pl = (kPair ? 2 * (r >> 1) * NT : r * NT) / (N * N);  // the same for the whole block at this r
    v[r] = pl < np ? src[i] : make_double2(0.0, 0.0);
    em[2 * pl] = max(em[2 * pl], oz::exp_field(v[r].x));
    em[2 * pl + 1] = max(em[2 * pl + 1], oz::exp_field(v[r].y));
  }
#pragma unroll
  for (int g = 0; g < G; ++g) {
    const unsigned m = oz::warp_max(em[g]);
    if (lane == 0) ered[w][g] = m;
  }
  __syncthreads();
  if (tid < G) {
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) m = max(m, ered[k][tid]);
    Eg[tid] = m;
  }
  __syncthreads();

  // 2. digits: dig[d][g][y][x] (with pairs: the two x-adjacent digits in one 32-bit store)
  if constexpr (kPair) {
#pragma unroll
    for (int r = 0; r < EPT; r += 2) {
      const int i = 2 * (tid + (r >> 1) * NT);
      const int pl = i / (N * N), rem = i % (N * N);
      const int y = rem / N, x = rem % N;
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        const int g = 2 * pl + ri;
        unsigned short d0[oz::S], d1[oz::S];
        oz::split(ri ? v[r].y : v[r].x, Eg[g], d0);
        oz::split(ri ? v[r + 1].y : v[r + 1].x, Eg[g], d1);
#pragma unroll
        for (int k = 0; k < oz::S; ++k)
          *reinterpret_cast<unsigned*>(dig + ((k * G + g) * N + y) * RS + x) = (unsigned)d0[k] | ((unsigned)d1[k] << 16);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < EPT; ++r) {
      const int i = tid + r * NT;
      const int pl = i / (N * N), rem = i % (N * N);
      const int y = rem / N, x = rem % N;
#pragma unroll
      for (int ri = 0; ri < 2; ++ri) {
        const int g = 2 * pl + ri;
        unsigned short d[oz::S];
        oz::split(ri ? v[r].y : v[r].x, Eg[g], d);
#pragma unroll
        for (int k = 0; k < oz::S; ++k) dig[((k * G + g) * N + y) * RS + x] = d[k];
      }
    }
  }
  __syncthreads();

  const int gq = lane >> 2, t4 = lane & 3;
  const int mi = lane >> 3, r8 = lane & 7;
  // every job of a warp has the output tile nt = w mod NTILE when NTILE divides the warp
  // count: its D2 fragments are then loaded once
  constexpr bool kBOnce = NW % NTILE == 0;
  uint32_t b[oz::S][KS][2];
  if (kBOnce) oz::load_b<KS>(b, a.ozb, w % NTILE, NTILE);
  // 3a. T_x: data rows (g, y), K = x'
  for (int job = w; job < MT * NTILE; job += NW) {
    const int mt = job / NTILE, nt = job % NTILE;
    const int g = mt / (N / 16), y0 = (mt % (N / 16)) * 16;
    if (!kBOnce) oz::load_b<KS>(b, a.ozb, nt, NTILE);
    int iacc[oz::S][4];
    oz::tile_levels<KS, false>(iacc, b, [&](int k, int ks) {
      return dig + ((k * G + g) * N + y0 + r8 + 8 * (mi & 1)) * RS + ks * 16 + 8 * (mi >> 1);
    });
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int lv[oz::S];
#pragma unroll
      for (int L = 0; L < oz::S; ++L) lv[L] = iacc[L][e];
      const int y = y0 + gq + 8 * (e >> 1), x = nt * 8 + 2 * t4 + (e & 1);
      acc64[(g * N + y) * N + x] = oz::combine(lv);
    }
  }
  __syncthreads();
  // 3b. T_y: data rows (g, x) by a transposed load of dig[.][g][y'][x], K = y'
  for (int job = w; job < MT * NTILE; job += NW) {
    const int mt = job / NTILE, nt = job % NTILE;
    const int g = mt / (N / 16), x0 = (mt % (N / 16)) * 16;
    if (!kBOnce) oz::load_b<KS>(b, a.ozb, nt, NTILE);
    int iacc[oz::S][4];
    oz::tile_levels<KS, true>(iacc, b, [&](int k, int ks) {
      return dig + ((k * G + g) * N + ks * 16 + 8 * (mi >> 1) + r8) * RS + x0 + 8 * (mi & 1);
    });
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int lv[oz::S];
#pragma unroll
      for (int L = 0; L < oz::S; ++L) lv[L] = iacc[L][e];
      const int x = x0 + gq + 8 * (e >> 1), y = nt * 8 + 2 * t4 + (e & 1);
      acc64[(g * N + y) * N + x] += oz::combine(lv);
    }
  }
  __syncthreads();

  // 4. FP64 values, coalesced store of T_xy x
  double2* dst = reinterpret_cast<double2*>(a.txy) + plane0 * N * N;
  for (int i = tid; i < np * N * N; i += NT) {
    const int pl = i / (N * N), rem = i % (N * N);
    // (the FP64 pipe is idle in this kernel: convert there)
    const double re = oz::to_double_hw(acc64[(2 * pl) * N * N + rem], oz::out_scale(a.oz_sD, Eg[2 * pl]));
    const double im = oz::to_double_hw(acc64[(2 * pl + 1) * N * N + rem], oz::out_scale(a.oz_sD, Eg[2 * pl + 1]));
    dst[i] = make_double2(re, im);
  }
}

// T_x + T_y of the FP64 path on the fifth-generation tensor cores (tcgen05), 32^3 lattices.
// One plane (a state component, N x N complex values) at a time; its exponent groups are the
// plane's real and imaginary parts.  The digit operand stacks the two axes into M = 128 rows,
// K = N:
//   rows g N + y       (g = re/im): the data lines along x  -> T_x x  [g][y][x = column]
//   rows 2N + g N + x:              the data lines along y  -> T_y x  [g][y = column][x]
// so one chain of MMAs against the D2 digits (B, N x K) forms both products.  Level L of the
// digit products (pairs k + l = L) accumulates in tensor-memory columns [L N, L N + N) of
// the plane's stage (exact FP32 integers, as in tile_levels); the levels are read back,
// combined in 64-bit integers per axis, summed and converted to FP64 once.
//
// Warp-specialised and persistent, one block per SM holding all 512 tensor-memory columns, so
// that the digit split, the MMAs and the read-back of different planes overlap:
//   consumers (the first kWsConsumerWarps warps): wait for mma_done[s], read the levels back
//     (warp w: lanes 32 (w % 4) .., its share of the columns), write the 64-bit sums into buffer
//     acc[s], release the stage (tmem_free[s]), then form T_x + T_y of the plane and store it;
//   producers (the next kWsProducerWarps warps): load a plane (one plane ahead), find its
//     exponent groups, write its digits into operand stage s = i % 2 (i: the block's plane
//     counter) and arrive on full[s];
//   issuer (the last warp, one thread): waits for full[s], issues the plane's 14 MMAs (7 data
//     digits x 2 K-steps, each against the stacked D2 digits) into the columns
//     [256 s, 256 s + 224) and commits to mma_done[s].
// A producer refills stage s (operand, scales) only after tmem_free[s].  Every wait is bounded
// (and gives up early once another role has given up): the block then records bit 4 in the
// error word, the issuer waits (bounded) for its last MMAs, and the tensor memory is freed.
#ifndef LISE_WS_PRODUCER_WARPS
#define LISE_WS_PRODUCER_WARPS 8
#endif
#ifndef LISE_WS_CONSUMER_WARPS
#define LISE_WS_CONSUMER_WARPS 8
#endif
// (measured on 32^3 x 2048, ms per launch: 8 producer + 8 consumer warps 2.02, 4 + 8 2.14, 8 + 4 2.50,
// 8 + 16 2.53)
constexpr int kWsProducerWarps = LISE_WS_PRODUCER_WARPS;  // 4 or 8
constexpr int kWsConsumerWarps = LISE_WS_CONSUMER_WARPS;  // 4, 8 or 16 (whole lane quadrants)
static_assert((kWsProducerWarps == 4 || kWsProducerWarps == 8) &&
                  (kWsConsumerWarps == 4 || kWsConsumerWarps == 8 || kWsConsumerWarps == 16),
              "role split");
constexpr int kWsThreads = 32 * (kWsConsumerWarps + kWsProducerWarps + 1);
template <int N>
struct TcPlanes {
  static_assert(N == 32, "two axes x two parts x N lines fill the 128 rows of one MMA only at N = 32");
  static constexpr int M = 4 * N, K = N;
  static constexpr int LBO = 128, SBO = (K / 8) * 128;  // core-matrix strides (bytes), K-major
  static constexpr int A_BYTES = M * K * 2, B_BYTES = N * K * 2;  // one digit of each operand
  static constexpr int AP = N + 1;                                 // padded row of the 64-bit sums
  static constexpr size_t acc_elems = (size_t)2 * 2 * N * AP;      // [T_x / T_y][g][N][AP]
  static constexpr size_t a_off = 0, b_off = (size_t)2 * oz::S * A_BYTES;  // two operand stages
  static constexpr size_t acc_off = b_off + (size_t)oz::S * B_BYTES;
  static constexpr size_t smem = acc_off + 2 * acc_elems * 8;      // two sums buffers
  static constexpr uint32_t TMEM_COLS = 512;  // two stages of S N <= 256 columns
  // word offset of the core-matrix D2 table behind the mma.sync fragment table
  static constexpr size_t table_offset = (size_t)oz::S * (N / 8) * (N / 16) * 32 * 2;
};
// byte offset of element (row, k) of a K-major core-matrix operand with K = 32
__device__ __forceinline__ int tc_off(int row, int k) {
  return (row >> 3) * TcPlanes<32>::SBO + (k >> 3) * TcPlanes<32>::LBO + (row & 7) * 16 + (k & 7) * 2;
}

template <int N>
__global__ void __launch_bounds__(kWsThreads, 1) k_planes_tc(PlanesArgs a) {
  static_assert(kWsThreads <= 1024, "block size");
  using P = TcPlanes<N>;
  constexpr int S = oz::S, AP = P::AP;
  constexpr int NP = 32 * kWsProducerWarps, NC = 32 * kWsConsumerWarps;  // producer, consumer threads
  constexpr int BAR_P = 1, BAR_C = 2;                                      // their named barriers
  extern __shared__ __align__(128) unsigned char smem_raw[];  // (no-swizzle operands need 16 bytes)
  unsigned char* sA = smem_raw + P::a_off;  // [2 stages][S][M rows][K], core-matrix layout
  unsigned char* sB = smem_raw + P::b_off;  // [S][N][K], core-matrix layout
  long long* accbuf = reinterpret_cast<long long*>(smem_raw + P::acc_off);  // [2][T_x / T_y][g][N][AP]
  __shared__ __align__(8) uint64_t full[2], mma_done[2], tmem_free[2];
  __shared__ uint32_t tslot;
  __shared__ unsigned ered[2][kWsProducerWarps][2];  // per stage: each producer warp's exponent maxima
  __shared__ unsigned Es[2][2];                      // per stage: the plane's exponent fields (re, im)
  __shared__ volatile int stop;                      // a role gave up: the others stop waiting
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  // the D2 digits, once per block (the table is stored in the core-matrix layout)
  const uint4* tb = reinterpret_cast<const uint4*>(a.ozb + P::table_offset);
  for (int i = tid; i < S * P::B_BYTES / 16; i += kWsThreads) reinterpret_cast<uint4*>(sB)[i] = tb[i];
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      um::mbar_init(&full[s], NP);
      um::mbar_init(&mma_done[s], 1);
      um::mbar_init(&tmem_free[s], 1);
    }
    stop = 0;
  }
  if (w == 0) um::alloc(&tslot, P::TMEM_COLS);
  um::fence_proxy_async();
  um::fence_before();
  __syncthreads();
  um::fence_after();
  const uint32_t tmem = tslot;
  const long limit = wait_limit(a.wait_polls);
  const long n_local = (a.n_planes - blockIdx.x + gridDim.x - 1) / gridDim.x;  // this block's planes
  auto give_up = [&]() {
    if (!stop) {
      stop = 1;
      if (a.err) atomicOr(a.err, 4);
    }
  };

  if (w >= kWsConsumerWarps && w < kWsConsumerWarps + kWsProducerWarps) {
    // ---------------------------------------------------------------- producers
    const int pt = tid - NC, pw = pt >> 5;
    // VB = 256 / NP 2 x 2 blocks per thread: the blocks of virtual threads vt = pt + NP j of a
    // 256-thread layout, an 8 x 8 tile per 16 lanes and two tiles per virtual warp (lane bits:
    // a = x pair, b = y pair, c = tile), so that the digit stores hit 32 distinct banks
    constexpr int VB = 256 / NP;
    int bx0[VB], by0[VB], blc[VB];
#pragma unroll
    for (int j = 0; j < VB; ++j) {
      const int vt = pt + NP * j, vw = vt >> 5, vl = vt & 31;
      blc[j] = vl >> 4;
      bx0[j] = 8 * (2 * (vw & 1) + blc[j]) + 2 * (vl & 3);
      by0[j] = 8 * (vw >> 1) + 2 * ((vl >> 2) & 3);
    }
    const double2* src0 = a.xr ? reinterpret_cast<const double2*>(a.xr) : a.x;
    double2 vn[VB][2][2];  // [j][dy][dx], the next plane's values (loaded one plane ahead)
    auto load_plane = [&](long pl) {
#pragma unroll
      for (int j = 0; j < VB; ++j)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx)
            vn[j][dy][dx] = pl < a.n_planes ? src0[pl * N * N + (by0[j] + dy) * N + bx0[j] + dx] : make_double2(0.0, 0.0);
    };
    load_plane(blockIdx.x);
    for (long i = 0; i < n_local; ++i) {
      const int s = (int)(i & 1);
      const uint32_t u = (uint32_t)(i >> 1);
      double2 v[VB][2][2];
      unsigned e0 = 0, e1 = 0;
#pragma unroll
      for (int j = 0; j < VB; ++j)
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            v[j][dy][dx] = vn[j][dy][dx];
            e0 = max(e0, oz::exp_field(v[j][dy][dx].x));
            e1 = max(e1, oz::exp_field(v[j][dy][dx].y));
          }
      load_plane(blockIdx.x + (i + 1) * gridDim.x);  // in flight through this plane's digit split
      e0 = oz::warp_max(e0);
      e1 = oz::warp_max(e1);
      if (lane == 0) {
        ered[s][pw][0] = e0;
        ered[s][pw][1] = e1;
      }
      // stage s is free once the consumers have released it (two planes back)
      bool ok = i < 2 || um::mbar_wait_or(&tmem_free[s], (u - 1) & 1u, limit, &stop);
      if (!um::bar_and(BAR_P, NP, ok)) {  // (also makes every warp's ered visible)
        give_up();
        break;
      }
      unsigned Eg[2] = {0, 0};
#pragma unroll
      for (int k = 0; k < kWsProducerWarps; ++k) {
        Eg[0] = max(Eg[0], ered[s][k][0]);
        Eg[1] = max(Eg[1], ered[s][k][1]);
      }
      if (pt == 0) {
        Es[s][0] = Eg[0];
        Es[s][1] = Eg[1];
      }
      unsigned char* sAs = sA + (size_t)s * S * P::A_BYTES;
      // digits into both row blocks (the lanes of one store cover one core matrix's 32 words:
      // rows alternate with the tile bit so that the two tiles of a warp use different rows)
#pragma unroll
      for (int j = 0; j < VB; ++j)
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          unsigned short d[2][2][S];
#pragma unroll
          for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) oz::split(g ? v[j][dy][dx].y : v[j][dy][dx].x, Eg[g], d[dy][dx]);
#pragma unroll
          for (int st = 0; st < 2; ++st) {
            const int o = st ^ blc[j];  // which row (dy for T_x, dx for T_y) this store covers
            const int ox = tc_off(g * N + by0[j] + o, bx0[j]);          // T_x row (g, y), k = x pair
            const int oy = tc_off(2 * N + g * N + bx0[j] + o, by0[j]);  // T_y row (g, x), k = y pair
#pragma unroll
            for (int k = 0; k < S; ++k) {
              const unsigned px0 = (unsigned)d[0][0][k] | ((unsigned)d[0][1][k] << 16);
              const unsigned px1 = (unsigned)d[1][0][k] | ((unsigned)d[1][1][k] << 16);
              const unsigned py0 = (unsigned)d[0][0][k] | ((unsigned)d[1][0][k] << 16);
              const unsigned py1 = (unsigned)d[0][1][k] | ((unsigned)d[1][1][k] << 16);
              *reinterpret_cast<unsigned*>(sAs + k * P::A_BYTES + ox) = o ? px1 : px0;
              *reinterpret_cast<unsigned*>(sAs + k * P::A_BYTES + oy) = o ? py1 : py0;
            }
          }
        }
      um::fence_proxy_async();  // the digits (generic proxy) before the tensor core reads them
      um::mbar_arrive(&full[s]);
    }
  } else if (w == kWsConsumerWarps + kWsProducerWarps) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      long committed = 0;
      for (long i = 0; i < n_local; ++i) {
        const int s = (int)(i & 1);
        if (!um::mbar_wait_or(&full[s], (uint32_t)(i >> 1) & 1u, limit, &stop)) {
          give_up();
          break;
        }
        um::fence_after();
        // descriptors of the first core matrices; the others differ only in the start-address field
        // (shared-memory addresses are below 2^18: the 14-bit field of address / 16 never carries)
        const uint64_t ad0 = um::sdesc(um::su32(sA + (size_t)s * S * P::A_BYTES), P::LBO, P::SBO);
        const uint64_t bd0 = um::sdesc(um::su32(sB), P::LBO, P::SBO);
        const uint32_t d0 = tmem + 256u * s;
        // The D2 digits are stacked along the MMA's N (B row l N + n is digit l of row n), so
        // that one MMA of width (S - k) N multiplies data digit k by D2 digits 0 .. S - 1 - k and
        // adds pair (k, l) into the columns of level k + l: it starts at column k N.  Chain
        // k = 0 covers every level (its first K-step initialises them).  Each level receives
        // the same exact products in the same order as one MMA per digit pair would give.
#pragma unroll
        for (int k = 0; k < S; ++k)
#pragma unroll
          for (int ks = 0; ks < P::K / 16; ++ks)
            um::mma_bf16(d0 + k * N, ad0 + (uint64_t)((k * P::A_BYTES + ks * 2 * P::LBO) >> 4),
                         bd0 + (uint64_t)((ks * 2 * P::LBO) >> 4), um::idesc_bf16_f32(P::M, (S - k) * N),
                         (k > 0 || ks > 0) ? 1u : 0u);
        um::commit(&mma_done[s]);
        committed = i + 1;
      }
      // the last MMAs complete before the tensor memory is freed (at once when the consumers
      // have already waited for them), bounded
      if (committed > 0)
        um::mbar_wait(&mma_done[(committed - 1) & 1], (uint32_t)((committed - 1) >> 1) & 1u, kDrainPolls);
    }
  } else if (w < kWsConsumerWarps) {
    // ---------------------------------------------------------------- consumers
    // warp w reads lane quadrant q = w % 4 (N = 32: q = 2 ax + g) and CW columns from c0
    constexpr int CW = N / (kWsConsumerWarps / 4);
    const int q = w & 3, c0 = CW * (w >> 2);
    const int g = q & 1, ax = q >> 1;
    for (long i = 0; i < n_local; ++i) {
      const int s = (int)(i & 1);
      const uint32_t par = (uint32_t)(i >> 1) & 1u;
      const long pl = blockIdx.x + i * gridDim.x;
      // the MMAs are done; full[s] (already complete) orders the producers' scales before us
      bool ok = um::mbar_wait_or(&mma_done[s], par, limit, &stop) && um::mbar_wait_or(&full[s], par, limit, &stop);
      if (!um::bar_and(BAR_C, NC, ok)) {
        give_up();
        break;
      }
      um::fence_after();
      const int ps0 = oz::out_scale(a.oz_sD, Es[s][0]), ps1 = oz::out_scale(a.oz_sD, Es[s][1]);
      long long* acc = accbuf + (size_t)s * P::acc_elems;
      long long* dst = acc + (size_t)ax * 2 * N * AP;
#pragma unroll
      for (int h = 0; h < CW / 8; ++h) {
        uint32_t r[S][8];
#pragma unroll
        for (int L = 0; L < S; ++L) um::ld8(r[L], tmem + ((uint32_t)(32 * q) << 16) + 256u * s + L * N + c0 + 8 * h);
        um::wait_ld_deps<S>(r);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          unsigned lb[S];
#pragma unroll
          for (int L = 0; L < S; ++L) lb[L] = __float_as_uint(__uint_as_float(r[L][j]) + 12582912.0f);
          dst[(g * N + c0 + 8 * h + j) * AP + lane] = oz::combine_biased(lb);
        }
      }
      um::fence_before();
      um::bar_sync(BAR_C, NC);  // every consumer has read stage s and written its sums
      if (tid == 0) um::mbar_arrive(&tmem_free[s]);
      // T_xy = T_x + T_y of the plane, one rounding; coalesced complex128 stores
      const long long* accx = acc;
      const long long* accy = acc + 2 * N * AP;
      double2* out = reinterpret_cast<double2*>(a.txy) + pl * N * N;
      for (int idx = tid; idx < N * N; idx += NC) {
        const int y = idx / N, x = idx % N;
        const long long re = accx[(0 * N + x) * AP + y] + accy[(0 * N + y) * AP + x];
        const long long im = accx[(1 * N + x) * AP + y] + accy[(1 * N + y) * AP + x];
        out[idx] = make_double2(oz::to_double_hw(re, ps0), oz::to_double_hw(im, ps1));
      }
    }
  }
  um::fence_before();
  __syncthreads();
  um::fence_after();
  if (w == 0) um::dealloc(tmem, P::TMEM_COLS);
}

// T_x + T_y of the FP64 path on tcgen05 for 48^3 lattices.  One plane's lines per axis and part
// are 2 x 48 = 96 rows, so each axis is one MMA row block of M = 128 (rows g N + line; rows 96-127
// are not read back), and a plane's seven level accumulators (7 x 48 columns per axis) exceed the
// tensor memory of two stages: the output columns are taken in chunks, [0, 32) and [32, 48).  Unit
// (axis, chunk), four per plane, accumulates levels L = k + l of the chunk's w output columns in one
// tensor-memory stage of 7 w columns (two stages, columns [256 s, 256 s + 7 w)): per data digit k and
// K-step, one MMA of width (7 - k) w against the chunk's stacked D2 digits 0 .. 6 - k (B row l w + n'
// is digit l of the chunk's D2 row n'), starting at column k w.
// Roles (one persistent block per SM):
//   producers: load a plane, find its two exponent groups (re, im), wait until the MMAs of the
//     previous plane are complete (a_free), write the digits of both axes (A_x: rows (g, y), K = x;
//     A_y: rows (g, x), K = y) and arrive on a_full;
//   issuer: for each unit, waits for a_full (first unit of a plane) and for its stage (tmem_free),
//     issues the 21 MMAs, commits to mma_done[stage]; after a plane's four units commits to a_free;
//   consumers: for each unit, read the stage's levels back (warp w: lanes 32 (w % 4)..; the two
//     warps of lane quadrant 3 hold no data rows and only take part in the barriers), combine them
//     in 64-bit integers into the plane's sums (T_x assigned, then T_y added), release the stage;
//     after the plane's four units convert the sums (one FP64 rounding) and store T_xy.
// Level sums with up to seven pairs over K = 48 can exceed 2^22 (levels 5 and 6): those two are
// converted to integers by the FP32 unit's exact conversion, the others by the 1.5 * 2^23 bias.
// Every wait is bounded and gives up once another role has given up.
constexpr int kTccProducerWarps = 6, kTccConsumerWarps = 8;
constexpr int kTccThreads = 32 * (kTccConsumerWarps + kTccProducerWarps + 1);
template <int N>
struct TcPlanesC {
  static_assert(N == 48, "the chunked tensor-memory planes kernel is laid out for 48-point lines");
  static constexpr int K = N, KS = K / 16, R = 2 * N, NCH = 2;            // rows, chunks per axis
  // output-column chunks: [0, 32) and [32, 48)
  __host__ __device__ static constexpr int cw(int o) { return o == 0 ? 32 : 16; }
  __host__ __device__ static constexpr int c0(int o) { return o == 0 ? 0 : 32; }
  static constexpr int LBO = 128, SBO = (K / 8) * 128;                    // K-major core matrices
  static constexpr int DA = (R / 8) * SBO;                                 // one digit of one axis (96 rows)
  static constexpr int A_AXIS = oz::S * DA + (128 - R) / 8 * SBO;           // + the unread rows 96-127
  // [digit][cw(o) rows][K] per chunk, chunk 1 after chunk 0
  __host__ __device__ static constexpr int b_chunk_off(int o) { return o == 0 ? 0 : oz::S * 32 * K * 2; }
  static constexpr int B_BYTES = oz::S * N * K * 2;
  static constexpr int AP = N + 1;                                         // padded row of the sums
  static constexpr size_t a_off = 0, b_off = (size_t)2 * A_AXIS;
  static constexpr size_t acc_off = b_off + (size_t)B_BYTES;
  static constexpr size_t smem = acc_off + (size_t)2 * N * AP * 8;         // sums [g][y][AP]
  static constexpr uint32_t TMEM_COLS = 512;                               // two stages at 256 s
  static constexpr int UNITS = 2 * NCH;                                    // (axis, chunk) per plane
  // word offset of the chunked core-matrix D2 table behind the mma.sync fragment table
  static constexpr size_t table_offset = (size_t)oz::S * (N / 8) * (N / 16) * 32 * 2;
};
__device__ __forceinline__ int tcc_off(int row, int k) {
  return (row >> 3) * TcPlanesC<48>::SBO + (k >> 3) * TcPlanesC<48>::LBO + (row & 7) * 16 + (k & 7) * 2;
}

template <int N>
__global__ void __launch_bounds__(kTccThreads, 1) k_planes_tcc(PlanesArgs a) {
  using P = TcPlanesC<N>;
  constexpr int S = oz::S, AP = P::AP;
  constexpr int NP = 32 * kTccProducerWarps, NC = 32 * kTccConsumerWarps;
  constexpr int BAR_P = 1, BAR_C = 2;
  constexpr int BLK = (N / 2) * (N / 2) / NP;  // 2 x 2 blocks of the plane per producer thread
  static_assert((N / 2) * (N / 2) % NP == 0, "producer blocks");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned char* sA = smem_raw + P::a_off;   // [axis][digit][rows][K], core-matrix layout
  unsigned char* sB = smem_raw + P::b_off;   // [chunk][digit][16][K], core-matrix layout
  long long* acc = reinterpret_cast<long long*>(smem_raw + P::acc_off);  // [g][y][AP]
  __shared__ __align__(8) uint64_t a_full, a_free, mma_done[2], tmem_free[2];
  __shared__ uint32_t tslot;
  __shared__ unsigned ered[kTccProducerWarps][2];
  __shared__ unsigned Es[2][2];  // per plane parity: the plane's exponent fields (re, im)
  __shared__ volatile int stop;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;

  const uint4* tb = reinterpret_cast<const uint4*>(a.ozb + P::table_offset);
  for (int i = tid; i < P::B_BYTES / 16; i += kTccThreads) reinterpret_cast<uint4*>(sB)[i] = tb[i];
  if (tid == 0) {
    um::mbar_init(&a_full, NP);
    um::mbar_init(&a_free, 1);
    for (int s = 0; s < 2; ++s) {
      um::mbar_init(&mma_done[s], 1);
      um::mbar_init(&tmem_free[s], 1);
    }
    stop = 0;
  }
  if (w == 0) um::alloc(&tslot, P::TMEM_COLS);
  um::fence_proxy_async();
  um::fence_before();
  __syncthreads();
  um::fence_after();
  const uint32_t tmem = tslot;
  const long limit = wait_limit(a.wait_polls);
  const long n_local = (a.n_planes - blockIdx.x + gridDim.x - 1) / gridDim.x;
  auto give_up = [&]() {
    if (!stop) {
      stop = 1;
      if (a.err) atomicOr(a.err, 4);
    }
  };

  if (w >= kTccConsumerWarps && w < kTccConsumerWarps + kTccProducerWarps) {
    // ---------------------------------------------------------------- producers
    const int pt = tid - NC, pw = pt >> 5;
    const double2* src0 = a.xr ? reinterpret_cast<const double2*>(a.xr) : a.x;
    for (long i = 0; i < n_local; ++i) {
      const long pl = blockIdx.x + i * gridDim.x;
      const double2* src = src0 + pl * N * N;
      double2 v[BLK][2][2];
      int by[BLK], bx[BLK];
      unsigned e0 = 0, e1 = 0;
#pragma unroll
      for (int b = 0; b < BLK; ++b) {
        const int blk = pt + NP * b;
        by[b] = 2 * (blk / (N / 2));
        bx[b] = 2 * (blk % (N / 2));
#pragma unroll
        for (int dy = 0; dy < 2; ++dy)
#pragma unroll
          for (int dx = 0; dx < 2; ++dx) {
            v[b][dy][dx] = src[(by[b] + dy) * N + bx[b] + dx];
            e0 = max(e0, oz::exp_field(v[b][dy][dx].x));
            e1 = max(e1, oz::exp_field(v[b][dy][dx].y));
          }
      }
      e0 = oz::warp_max(e0);
      e1 = oz::warp_max(e1);
      if (lane == 0) {
        ered[pw][0] = e0;
        ered[pw][1] = e1;
      }
      // the previous plane's MMAs have read the operand
      bool ok = i < 1 || um::mbar_wait_or(&a_free, (uint32_t)((i - 1) & 1), limit, &stop);
      if (!um::bar_and(BAR_P, NP, ok)) {  // (also makes every warp's ered visible)
        give_up();
        break;
      }
      unsigned Eg[2] = {0, 0};
#pragma unroll
      for (int k = 0; k < kTccProducerWarps; ++k) {
        Eg[0] = max(Eg[0], ered[k][0]);
        Eg[1] = max(Eg[1], ered[k][1]);
      }
      if (pt == 0) {
        Es[i & 1][0] = Eg[0];
        Es[i & 1][1] = Eg[1];
      }
#pragma unroll
      for (int b = 0; b < BLK; ++b)
#pragma unroll
        for (int g = 0; g < 2; ++g) {
          unsigned short d[2][2][S];
#pragma unroll
          for (int dy = 0; dy < 2; ++dy)
#pragma unroll
            for (int dx = 0; dx < 2; ++dx) oz::split(g ? v[b][dy][dx].y : v[b][dy][dx].x, Eg[g], d[dy][dx]);
#pragma unroll
          for (int o = 0; o < 2; ++o) {
            const int ox = tcc_off(g * N + by[b] + o, bx[b]);  // A_x row (g, y), k = x pair
            const int oy = tcc_off(g * N + bx[b] + o, by[b]);  // A_y row (g, x), k = y pair
#pragma unroll
            for (int k = 0; k < S; ++k) {
              *reinterpret_cast<unsigned*>(sA + k * P::DA + ox) = (unsigned)d[o][0][k] | ((unsigned)d[o][1][k] << 16);
              *reinterpret_cast<unsigned*>(sA + P::A_AXIS + k * P::DA + oy) =
                  (unsigned)d[0][o][k] | ((unsigned)d[1][o][k] << 16);
            }
          }
        }
      um::fence_proxy_async();  // the digits (generic proxy) before the tensor core reads them
      um::mbar_arrive(&a_full);
    }
  } else if (w == kTccConsumerWarps + kTccProducerWarps) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      long nfree = 0;        // commits to a_free so far
      bool pending = false;  // MMAs issued since the last commit to a_free
      bool ok = true;
      for (long i = 0; i < n_local && ok; ++i) {
        if (!um::mbar_wait_or(&a_full, (uint32_t)(i & 1), limit, &stop)) {
          give_up();
          break;
        }
        um::fence_after();
#pragma unroll
        for (int u = 0; u < P::UNITS; ++u) {
          const long j = i * P::UNITS + u;
          const int s = (int)(j & 1), ax = u / P::NCH, o = u % P::NCH;
          if (j >= 2 && !um::mbar_wait_or(&tmem_free[s], (uint32_t)(((j >> 1) - 1) & 1), limit, &stop)) {
            give_up();
            ok = false;
            break;
          }
          um::fence_after();
          const uint32_t d0 = tmem + 256u * s;
          // descriptors of the unit's first core matrices; the others differ only in the start
          // address field (shared-memory addresses are below 2^18, so the 14-bit field of
          // address / 16 never carries into the next field)
          const uint64_t ad0 = um::sdesc(um::su32(sA + (size_t)ax * P::A_AXIS), P::LBO, P::SBO);
          const uint64_t bd0 = um::sdesc(um::su32(sB + P::b_chunk_off(o)), P::LBO, P::SBO);
          const int cw = P::cw(o);
#pragma unroll
          for (int k = 0; k < S; ++k)
#pragma unroll
            for (int ks = 0; ks < P::KS; ++ks)
              um::mma_bf16(d0 + k * cw, ad0 + (uint64_t)((k * P::DA + ks * 2 * P::LBO) >> 4),
                           bd0 + (uint64_t)((ks * 2 * P::LBO) >> 4), um::idesc_bf16_f32(128, (S - k) * cw),
                           (k > 0 || ks > 0) ? 1u : 0u);
          um::commit(&mma_done[s]);
          pending = true;
        }
        if (!ok) break;
        um::commit(&a_free);  // every MMA of the plane has read the operand
        ++nfree;
        pending = false;
      }
      // every MMA issued completes before the tensor memory is freed (a block that gave up in
      // the middle of a plane commits once more), bounded
      if (pending) {
        um::commit(&a_free);
        ++nfree;
      }
      if (nfree > 0) um::mbar_wait(&a_free, (uint32_t)((nfree - 1) & 1), kDrainPolls);
    }
  } else if (w < kTccConsumerWarps) {
    // ---------------------------------------------------------------- consumers
    const int q = w & 3, h = w >> 2;   // lane quadrant, column half of the chunk
    const int r = 32 * q + lane;       // data row (r < 96)
    const int g = r / N, line = r % N;
    for (long i = 0; i < n_local; ++i) {
      const long pl = blockIdx.x + i * gridDim.x;
      int ps0 = 0, ps1 = 0;
      bool ok = true;
      for (int u = 0; u < P::UNITS && ok; ++u) {
        const long j = i * P::UNITS + u;
        const int s = (int)(j & 1), ax = u / P::NCH, o = u % P::NCH;
        ok = um::mbar_wait_or(&mma_done[s], (uint32_t)((j >> 1) & 1), limit, &stop);
        // (the plane's operand is complete: a_full orders the producers' scales before us)
        if (ok && u == 0) ok = um::mbar_wait_or(&a_full, (uint32_t)(i & 1), limit, &stop);
        if (!um::bar_and(BAR_C, NC, ok)) {
          ok = false;
          break;
        }
        um::fence_after();
        if (u == 0) {
          ps0 = oz::out_scale(a.oz_sD, Es[i & 1][0]);
          ps1 = oz::out_scale(a.oz_sD, Es[i & 1][1]);
        }
        if (q < 3) {
          // this warp's half of the chunk: cw / 2 columns, 8 at a time
          const int cw = P::cw(o);
          for (int part = 0; part < cw / 16; ++part) {
            const int col = (cw / 2) * h + 8 * part;  // first column within the chunk
            uint32_t rv[S][8];
#pragma unroll
            for (int L = 0; L < S; ++L) um::ld8(rv[L], tmem + ((uint32_t)(32 * q) << 16) + 256u * s + L * cw + col);
            um::wait_ld_deps<S>(rv);
#pragma unroll
            for (int c = 0; c < 8; ++c) {
              unsigned lb[S];
#pragma unroll
              for (int L = 0; L < S; ++L) {
                const float f = __uint_as_float(rv[L][c]);
                lb[L] = L < 5 ? __float_as_uint(f + 12582912.0f) : (unsigned)__float2int_rn(f) + 0x4B400000u;
              }
              const long long T = oz::combine_biased(lb);
              const int n = P::c0(o) + col + c;
              if (ax == 0)
                acc[(g * N + line) * AP + n] = T;   // T_x[g][y = line][x = n]
              else
                acc[(g * N + n) * AP + line] += T;  // T_y[g][y = n][x = line]
            }
          }
        }
        um::fence_before();
        um::bar_sync(BAR_C, NC);  // every consumer has read stage s and written its sums
        if (tid == 0) um::mbar_arrive(&tmem_free[s]);
      }
      if (!ok) {
        give_up();
        break;
      }
      // T_xy = T_x + T_y of the plane, one rounding; coalesced complex128 stores
      double2* out = reinterpret_cast<double2*>(a.txy) + pl * N * N;
      for (int idx = tid; idx < N * N; idx += NC) {
        const int y = idx / N, x = idx % N;
        out[idx] = make_double2(oz::to_double_hw(acc[y * AP + x], ps0), oz::to_double_hw(acc[(N + y) * AP + x], ps1));
      }
      um::bar_sync(BAR_C, NC);  // the sums are read before the next plane's T_x is assigned
    }
  }
  um::fence_before();
  __syncthreads();
  um::fence_after();
  if (w == 0) um::dealloc(tmem, P::TMEM_COLS);
}

// T_z x on the tensor cores for one pencils batch (FP64 path, N % 16 == 0):
// operand xr[j][c] of this thread's site (z, xl); result T_z x into buf[(2j + c) CS + z TX + xl].
// Exponent groups: (state j, component c, re/im) over the block's (z, x) tile; data
// rows: columns col = group TX + xl of dig[d][col][z'], K = z'.
template <int N, int TX, int QB, int CS>
__device__ __forceinline__ void oz_pencils_tz(const double2 (&xr)[QB][2], double2* buf, unsigned short* dig,
                                              unsigned* ered, unsigned* Eg, const uint32_t* ozb, int sD, int z,
                                              int xl) {
  constexpr int NT = N * TX, NW = NT / 32, NE = QB * 4, RS = N + 8;
  constexpr int KS = N / 16, NTILE = N / 8, NCOL = NE * TX, MT = NCOL / 16;
  static_assert(NCOL % 16 == 0, "pencil columns");
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int g = 0; g < NE; ++g) {
    const double2 v = xr[g >> 2][(g >> 1) & 1];
    const unsigned m = oz::warp_max(oz::exp_field((g & 1) ? v.y : v.x));
    if (lane == 0) ered[w * NE + g] = m;
  }
  __syncthreads();
  if (tid < NE) {
    unsigned m = 0;
#pragma unroll
    for (int k = 0; k < NW; ++k) m = max(m, ered[k * NE + tid]);
    Eg[tid] = m;
  }
  __syncthreads();
#pragma unroll
  for (int g = 0; g < NE; ++g) {
    const double2 v = xr[g >> 2][(g >> 1) & 1];
    unsigned short d[oz::S];
    oz::split((g & 1) ? v.y : v.x, Eg[g], d);
#pragma unroll
    for (int k = 0; k < oz::S; ++k) dig[(k * NCOL + g * TX + xl) * RS + z] = d[k];
  }
  __syncthreads();
  const int gq = lane >> 2, t4 = lane & 3, mi = lane >> 3, r8 = lane & 7;
  double* out = reinterpret_cast<double*>(buf);
  constexpr bool kBOnce = NW % NTILE == 0;  // as in k_planes_oz
  uint32_t b[oz::S][KS][2];
  if (kBOnce) oz::load_b<KS>(b, ozb, w % NTILE, NTILE);
  for (int job = w; job < MT * NTILE; job += NW) {
    const int mt = job / NTILE, nt = job % NTILE;
    if (!kBOnce) oz::load_b<KS>(b, ozb, nt, NTILE);
    int iacc[oz::S][4];
    oz::tile_levels<KS, false>(iacc, b, [&](int k, int ks) {
      return dig + (k * NCOL + mt * 16 + r8 + 8 * (mi & 1)) * RS + ks * 16 + 8 * (mi >> 1);
    });
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      int lv[oz::S];
#pragma unroll
      for (int L = 0; L < oz::S; ++L) lv[L] = iacc[L][e];
      const int col = mt * 16 + gq + 8 * (e >> 1), zz = nt * 8 + 2 * t4 + (e & 1);
      const int g = col / TX, x2 = col % TX;
      // T_xy (already in the buffer) added in the integer domain
      double& o = out[2 * ((g >> 1) * CS + zz * TX + x2) + (g & 1)];
      o = oz::add_to_double(oz::combine(lv), o, oz::out_scale(sD, Eg[g]));
    }
  }
  __syncthreads();
}

// ----------------------------------------------------------------- pencils --
// Byte offset of the prefetch staging area in the pencils kernel's shared memory
// (after the FFT buffer, the twiddles and the kinetic factors), 128-byte aligned (the
// staging arrays are destinations of tensor-map copies).
template <typename T, int N, int TX, int QB>
__host__ __device__ constexpr int pencil_stage_offset() {
  return (((QB * 2 * (N * TX + (sizeof(T) == 8 ? 8 : 0)) + N) * (int)sizeof(T) + N * (int)sizeof(T) / 2) + 127) / 128 * 128;
}
// FP64 tensor-core path (lise_ozaki.cuh) on lattices with N % 16 == 0
template <typename R, int N>
__host__ __device__ constexpr bool pencil_oz() { return sizeof(R) == 8 && N % 16 == 0; }
// x-tile width of the pencils kernel: 4 on the FP64 tensor-core path (128-thread blocks, several
// resident per SM, so that blocks in their digit/tensor phase overlap others in their FP64
// epilogue) and for N not a multiple of 8, else 8
template <typename R, int N>
__host__ __device__ constexpr int pencil_tx_c() {
  return (pencil_oz<R, N>() || N % 8 != 0) ? 4 : 8;
}
template <typename T, int N, int TX, int QB>
__host__ __device__ constexpr int pencil_smem_bytes() {
  // staging only for the FP32 compute precision (see kPrefetch in k_pencils): the next
  // batch's operand and T_xy, and this batch's Q (complex128) and R (compute precision);
  // digit planes [7][QB * 4 * TX][N + 8] (bf16) for the FP64 tensor-core path
  return pencil_stage_offset<T, N, TX, QB>() +
         (sizeof(T) == 8 ? QB * 2 * N * TX * (16 + (int)sizeof(T) + 16 + (int)sizeof(T))
                         : (N % 16 == 0 ? oz::S * QB * 4 * TX * (N + 8) * 2 : 0));
}

// ST (FP32 compute precision, corrector mode only): the strict split of LISE_MIXED_STRICT --
// R and p - c in complex128 (units of h/48), y_{n+1} = Q + k1 m' and p - c = R - 17 m' in
// FP64 from the exact FP64 value of m', densities of y_{n+1} from its FP64 values.
// Block (bx of nbx) of group g of the evolution described by a.
template <typename R, int N, int TX, int QB, int MODE, bool ST>
__device__ __forceinline__ void pencils_body(const PencilArgs& a, const int g, const int bx, const int nbx) {
  using T = typename Cx<R>::T;
  constexpr int NT = N * TX;
  // one component block [z][x] in shared memory; for 8-byte elements the blocks are
  // padded by 64 bytes so the four blocks a warp touches fall on different banks
  constexpr int CS = N * TX + (sizeof(T) == 8 ? 8 : 0);
  constexpr int LINES = QB * 2 * TX;   // z-lines per batch
  extern __shared__ __align__(128) unsigned char smem_raw[];
  T* buf = reinterpret_cast<T*>(smem_raw);  // [QB][2][N][TX]
  T* tw = buf + QB * 2 * CS;
  R* hz = reinterpret_cast<R*>(tw + N);
  // prefetch staging for the next batch, [QB * 2][NT] per array: the operand as
  // stored (complex128, or the compute precision when a.xr is set) and T_xy
  double2* xstage = reinterpret_cast<double2*>(smem_raw + pencil_stage_offset<T, N, TX, QB>());
  T* tstage = reinterpret_cast<T*>(xstage + QB * 2 * NT);
  double2* qstage = reinterpret_cast<double2*>(tstage + QB * 2 * NT);  // Q then R of this batch
  T* rstage = reinterpret_cast<T*>(qstage + QB * 2 * NT);
  constexpr bool kOz = pencil_oz<R, N>();
  unsigned short* dig = reinterpret_cast<unsigned short*>(smem_raw + pencil_stage_offset<T, N, TX, QB>());
  __shared__ unsigned oz_e[(N * TX / 32 + 1) * QB * 4];
  const T* twg = reinterpret_cast<const T*>(a.tw);
  const R* hg = reinterpret_cast<const R*>(a.hz);
  for (int i = threadIdx.x; i < N; i += NT) {
    tw[i] = twg[i];
    hz[i] = hg[i];
  }
  const long nxyz = (long)N * N * N;
  constexpr int TILES_X = N / TX;
  const int y = bx / TILES_X;
  const int x0 = (bx % TILES_X) * TX;
  const int z = threadIdx.x / TX, xl = threadIdx.x % TX;
  const long site = ((long)z * N + y) * N + x0 + xl;
  const int q_begin = g * a.qg;
  const int q_end = min(a.n_qp, q_begin + a.qg);
  double Wv = 0.0;
  double2 Dv = make_double2(0.0, 0.0);
  if (MODE != M_ENERGY) {
    Wv = a.W[site];
    Dv = a.D[site];
  }
  const T* txy = reinterpret_cast<const T*>(a.txy);
  const R Wr = (R)Wv;
  const T Dr = to_r<R>(Dv);
  double sn = 0.0, sr = 0.0, si = 0.0;
  DensF dF;  // FP32 operands (mixed path)
  // step-size coefficients of the ABM epilogues, once per thread:
  //   corrector  y_{n+1} = Q + kc1 m',  p - c = R - kc2 m'
  //   predictor  Y = sum y?c y'_?,  R = sum r?c y'_?  (see M_DERIV_PREDICT)
  // In FP64, R and p - c are kept in units of h/48 (R = 68 y'_{n+1} - 102 y'_n + ..., the
  // exact integer-coefficient sum, p - c = R - 17 m'): the scale h/48 then enters once, where
  // m is formed, instead of once per stored value.
  constexpr bool kCor = MODE == M_CORRECT, kPred = MODE == M_DERIV_PREDICT;
  const R kc2 = kCor ? (sizeof(R) == 8 ? R(17) : (R)(17.0 / 48.0 * a.h)) : R(0),
          kc1 = kCor ? (R)(161.0 / 170.0 * 17.0 / 48.0 * a.h) : R(0);
  const R h48 = kPred ? (R)(a.h / 48.0) : R(0), c161_ = (R)(161.0 / 170.0), c9_ = (R)(9.0 / 170.0);
  const R y0c = h48 * (c161_ * R(51) + c9_ * R(119)), y1c = h48 * (c161_ * R(3) - c9_ * R(99)),
          y2c = h48 * (c161_ + c9_ * R(69)), y3c = h48 * (-c9_ * R(17));
  const R r0c = h48 * R(68), r1c = h48 * R(-102), r2c = h48 * R(68), r3c = h48 * R(-17);
  const R c161h = c161_ * h48;
  auto base = [](int l) { return (l / TX) * CS + (l % TX); };
  // The prefetch pays in the memory-bound mixed path; the FP64 path is FP64-pipe bound and
  // keeps its registers for occupancy (plain loads).  Staging by the tensor memory
  // accelerator: one thread copies the batch's box [2 QB planes][N z][TX x] of the operand
  // and of T_xy (and, in the corrector, of Q and R) into shared memory; completion on an
  // mbarrier per staged pair (bounded waits: a wait that runs out sets bit 4 of the error word).
  constexpr bool kPrefetch = sizeof(R) == 4;
  __shared__ __align__(8) uint64_t mb_stage[2];  // [0] operand + T_xy, [1] Q + R
  uint32_t ph_x = 0, ph_q = 0;
  const uint32_t bytes_x = 2u * QB * NT * ((a.xr ? (uint32_t)sizeof(T) : 16u) + (uint32_t)sizeof(T));
  const uint32_t bytes_q = 2u * QB * NT * (16u + (ST ? 0u : (uint32_t)sizeof(T)));  // Q (and R unless ST)
  // tensor copies need 128-byte aligned destinations: checked, never assumed (a block whose
  // staging is misaligned copies nothing and reports through the error word)
  const bool stage_ok = (um::su32(xstage) & 127u) == 0;
  // A wait that runs out sets bit 4 of the error word and `failed`; the block then stops at
  // its next barrier (__syncthreads_or, so all its threads stop together), consumes no more
  // staged data and issues no further copy.  Thread 0, which issues the copies, first waits
  // (bounded) for the copy it gave up on, and before the block exits for any copy still in
  // flight, so that no copy lands in the shared memory of a block that has exited.
  bool failed = kPrefetch && !stage_ok;
  bool pend[2] = {false, false};  // thread 0: copies issued on stage k that have not completed
  auto prefetch = [&](int qb) {
    if (threadIdx.x == 0 && stage_ok) {
      um::fence_proxy_async();  // the staging reads of the previous batch before the copies
      um::mbar_expect_tx(&mb_stage[0], bytes_x);
      um::tma_load_4d(xstage, &a.tm_x, 2 * x0, y, 0, 2 * qb, &mb_stage[0]);
      um::tma_load_4d(tstage, &a.tm_t, 2 * x0, y, 0, 2 * qb, &mb_stage[0]);
      pend[0] = true;
    }
  };
  auto wait_stage = [&](int k, uint32_t& ph) {
    if (stage_ok) {
      if (!um::mbar_wait(&mb_stage[k], ph, wait_limit(a.wait_polls))) {
        failed = true;
        if (a.err) atomicOr(a.err, 4);
        if (threadIdx.x == 0) um::mbar_wait(&mb_stage[k], ph, kDrainPolls);
      }
      if (threadIdx.x == 0) pend[k] = false;
    }
    ph ^= 1u;
  };
  if constexpr (kPrefetch) {
    if (!stage_ok && threadIdx.x == 0 && a.err) atomicOr(a.err, 4);
    if (threadIdx.x == 0) {
      um::mbar_init(&mb_stage[0], 1);
      um::mbar_init(&mb_stage[1], 1);
    }
    if (q_begin < q_end) prefetch(q_begin);
  }
  __syncthreads();

  for (int qb0 = q_begin; qb0 < q_end; qb0 += QB) {
    double eta_acc[QB];
#pragma unroll
    for (int j = 0; j < QB; ++j) eta_acc[j] = 0.0;
    T xr[QB][2];  // the operand in compute precision (FP64 values are reloaded where needed)
    T tr[QB][2];  // T_xy of this batch (prefetch path)
    if constexpr (kPrefetch) {
      wait_stage(0, ph_x);
#pragma unroll
      for (int j = 0; j < QB; ++j) {
        const int q = qb0 + j;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int si_ = (2 * j + c) * NT + threadIdx.x;
          T v = T{R(0), R(0)}, t = T{R(0), R(0)};
          if (q < q_end) {
            v = a.xr ? reinterpret_cast<const T*>(xstage)[si_] : to_r<R>(xstage[si_]);
            t = tstage[si_];
          }
          xr[j][c] = v;
          tr[j][c] = t;
          buf[(2 * j + c) * CS + z * TX + xl] = v;
        }
      }
      // (also orders the staging reads above before the next batch's copies)
      if (__syncthreads_or(failed)) break;
      if constexpr (MODE == M_CORRECT) {
        // this batch's Q and R (read in the epilogue, after the line transforms)
        if (threadIdx.x == 0 && stage_ok) {
          um::fence_proxy_async();
          um::mbar_expect_tx(&mb_stage[1], bytes_q);
          um::tma_load_4d(qstage, &a.tm_q, 2 * x0, y, 0, 2 * qb0, &mb_stage[1]);
          if constexpr (!ST) um::tma_load_4d(rstage, &a.tm_r, 2 * x0, y, 0, 2 * qb0, &mb_stage[1]);
          pend[1] = true;
        }
      }
      // the staging buffers are free again: fetch the next batch while this one computes
      if (qb0 + QB < q_end) prefetch(qb0 + QB);
    } else {
#pragma unroll
      for (int j = 0; j < QB; ++j) {
        const int q = qb0 + j;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const long gi = (long)(2 * q + c) * nxyz + site;
          const T v = q < q_end ? (a.xr ? reinterpret_cast<const T*>(a.xr)[gi] : to_r<R>(a.x[gi])) : T{R(0), R(0)};
          xr[j][c] = v;
          if (!kOz) buf[(2 * j + c) * CS + z * TX + xl] = v;
          else buf[(2 * j + c) * CS + z * TX + xl] = q < q_end ? txy[gi] : T{R(0), R(0)};
        }
      }
      if (!kOz) __syncthreads();
    }
    if constexpr (kOz) {
      oz_pencils_tz<N, TX, QB, CS>(xr, buf, dig, oz_e, oz_e + (NT / 32) * QB * 4, a.ozb, a.oz_sD, z, xl);
    } else {
      fft_lines<N, -1, R, LINES, NT>(buf, base, TX, tw, [&](int, int k, T v) {
        R f = hz[k];
        return T{v.x * f, v.y * f};
      });
      fft_lines<N, +1, R, LINES, NT>(buf, base, TX, tw, Identity());
    }
    if constexpr (kPrefetch && MODE == M_CORRECT) wait_stage(1, ph_q);  // Q, R of this batch

#pragma unroll
    for (int j = 0; j < QB; ++j) {
      const int q = qb0 + j;
      if (q >= q_end) break;
      const long iu = (long)(2 * q) * nxyz + site, iv = iu + nxyz;
      // FP64 tensor-core path: T_z + T_xy already summed (integer domain) in the buffer
      const T Tu = kOz ? buf[(2 * j) * CS + z * TX + xl] : cadd(buf[(2 * j) * CS + z * TX + xl], kPrefetch ? tr[j][0] : txy[iu]);
      const T Tv = kOz ? buf[(2 * j + 1) * CS + z * TX + xl] : cadd(buf[(2 * j + 1) * CS + z * TX + xl], kPrefetch ? tr[j][1] : txy[iv]);
      if (MODE == M_ENERGY) {
        const double2 v = a.x[iv];
        const double2 tv = to_d(Tv);
        sn = fma(v.x, tv.x, fma(v.y, tv.y, sn));
        continue;
      }
      // H x = [[h, Delta], [Delta*, -h*]] x with h = T + W (W real, T real-symmetric);
      // with trivial-phase removal (Eq. sp_en) the generator is H - eta_q.
      // The FP64 tensor-core path reloads the operand (an L2 hit) rather than keeping it in
      // registers across the digit products.  The epilogue's loads bypass L1 (ld.global.cg;
      // 32^3 x 2048 FP64: 5.38 -> 5.34 ms per launch).
      auto opnd = [&](long i) -> T {
        return a.xr ? __ldcg(reinterpret_cast<const T*>(a.xr) + i) : to_r<R>(__ldcg(a.x + i));
      };
      const T u = kOz ? opnd(iu) : xr[j][0], v = kOz ? opnd(iv) : xr[j][1];
      const R w = a.eta ? Wr - (R)a.eta[q] : Wr;
      const R w2 = a.eta ? Wr + (R)a.eta[q] : Wr;  // -(h + eta) on the v component
      const T d = Dr;
      // one FMA chain per real part (3 FMA after the kinetic sum)
      const T hu = T{fmx(w, u.x, fmx(d.x, v.x, fmx(-d.y, v.y, Tu.x))), fmx(w, u.y, fmx(d.x, v.y, fmx(d.y, v.x, Tu.y)))};
      const T hv = T{fmx(-w2, v.x, fmx(d.x, u.x, fmx(d.y, u.y, -Tv.x))), fmx(-w2, v.y, fmx(d.x, u.y, fmx(-d.y, u.x, -Tv.y)))};
      if (MODE == M_ETA) {
        const double2 du = to_d(u), dv = to_d(v), Hu_ = to_d(hu), Hv_ = to_d(hv);
        eta_acc[j] += (du.x * Hu_.x + du.y * Hu_.y) + (dv.x * Hv_.x + dv.y * Hv_.y);
        continue;
      }
      const T fur = T{hu.y, -hu.x}, fvr = T{hv.y, -hv.x};  // -i H x, compute precision
      const double2 Hu = to_d(hu), Hv = to_d(hv);
      const double2 fu = make_double2(Hu.y, -Hu.x), fv = make_double2(Hv.y, -Hv.x);  // -i H x

      T* dslot = reinterpret_cast<T*>(a.dslot);
      if (MODE == M_RHS) {
        if (a.out) {
          a.out[iu] = fu;
          a.out[iv] = fv;
        }
        if (dslot) {
          dslot[iu] = fur;
          dslot[iv] = fvr;
        }
      } else if (MODE == M_TAYLOR_FIRST) {
        if (dslot) {
          dslot[iu] = fur;
          dslot[iv] = fvr;
        }
        const double2 tu = dmul(a.coef, Hu), tv = dmul(a.coef, Hv);
        a.out[iu] = tu;
        a.out[iv] = tv;
        a.acc[iu] = dadd(a.x[iu], tu);
        a.acc[iv] = dadd(a.x[iv], tv);
      } else if (MODE == M_TAYLOR) {
        const double2 tu = dmul(a.coef, Hu), tv = dmul(a.coef, Hv);
        a.out[iu] = tu;
        a.out[iv] = tv;
        const double2 au = dadd(a.acc[iu], tu), av = dadd(a.acc[iv], tv);
        a.acc[iu] = au;
        a.acc[iv] = av;
        if (a.dens) dens_acc(au, av, sn, sr, si);
      } else if (MODE == M_CORRECT) {
        // Eq. c and Eq. y through Q, R:  y_{n+1} = Q + k1 m',  p - c = R - k2 m'
        const R k2 = kc2, k1 = kc1;
        T yo[2];          // y_{n+1} in the compute precision, for its densities
        double2 yd[2];    // (ST: the FP64 values)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const long i = c ? iv : iu;
          const T f = c ? fvr : fur;
          const int si_ = (2 * j + c) * NT + threadIdx.x;
          double2 yn;
          if constexpr (ST) {
            // FP64 history arithmetic from the exact FP64 value of m'
            const double2 fd = to_d(f), qv = kPrefetch ? qstage[si_] : a.q[i];
            const double2 rr = reinterpret_cast<const double2*>(a.r)[i];
            // (R and p - c in units of h/48, as in the FP64 path: p - c = R - 17 m')
            const double k1d = 161.0 / 170.0 * 17.0 / 48.0 * a.h;
            yn = make_double2(fma(k1d, fd.x, qv.x), fma(k1d, fd.y, qv.y));
            reinterpret_cast<double2*>(a.pc)[i] = make_double2(fma(-17.0, fd.x, rr.x), fma(-17.0, fd.y, rr.y));
            yd[c] = yn;
          } else {
            const T rr = kPrefetch ? rstage[si_] : __ldcg(reinterpret_cast<const T*>(a.r) + i);
            if constexpr (sizeof(R) == 8) {
              const double2 qv = __ldcg(a.q + i);
              yn = make_double2(fma((double)k1, (double)f.x, qv.x), fma((double)k1, (double)f.y, qv.y));
            } else {
              yn = dadd(kPrefetch ? qstage[si_] : a.q[i], to_d(T{k1 * f.x, k1 * f.y}));
            }
            reinterpret_cast<T*>(a.pc)[i] = T{rr.x - k2 * f.x, rr.y - k2 * f.y};
          }
          a.ynew[i] = yn;
          yo[c] = to_r<R>(yn);
        }
        if constexpr (ST)
          dens_acc(yd[0], yd[1], sn, sr, si);
        else if constexpr (sizeof(R) == 4)
          dens_acc(yo[0], yo[1], dF);
        else
          dens_acc(yo[0], yo[1], sn, sr, si);
      } else if (MODE == M_DERIV_PREDICT) {
        // y'_{n+1}; then Eq. p and Eq. m of step n+2 and that step's Q, R:
        //   pt = h/48 (119 y'_{n+1} - 99 y'_n + 69 y'_{n-1} - 17 y'_{n-2})
        //   ct = h/48 (51 y'_{n+1} + 3 y'_n + y'_{n-1}),  hf = (y_{n+1} + y_n)/2
        //   m = hf + pt - (161/170) pc,  Q = hf + (161/170) ct + (9/170) pt,  R = pt - ct.
        // FP64: from the exact integer sums sp = 48 pt / h and sr = 48 R / h (pred_sums),
        //   P = hf + pt (Eq. p),  Q = P - (161/170) R,  m = P - (161/170) pc  (Eq. m),
        // with R and pc kept in units of h/48.  FP32 compute precision: Y = (161/170) ct +
        // (9/170) pt and R directly from the derivatives, Q = hf + Y and m = Q + (161/170)(R - pc)
        // (as 1 - 9/170 = 161/170, m - Q = (161/170)(pt - ct - pc)).
        const R c161 = (R)(161.0 / 170.0);
        T mo[2];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const long i = c ? iv : iu;
          const T f = c ? fvr : fur;
          dslot[i] = f;
          const T e0 = __ldcg(reinterpret_cast<const T*>(a.d0) + i), e1 = __ldcg(reinterpret_cast<const T*>(a.d1) + i),
                  e2 = __ldcg(reinterpret_cast<const T*>(a.d2) + i);
          const T pcv = __ldcg(reinterpret_cast<const T*>(a.pc) + i);
          const double2 xv = __ldcg(a.x + i), y0v = __ldcg(a.y0 + i);
          T Rv, mv;
          double2 qv;
          if constexpr (sizeof(R) == 8) {
            double spx, srx, spy, sry;
            pred_sums(f.x, e0.x, e1.x, e2.x, spx, srx);
            pred_sums(f.y, e0.y, e1.y, e2.y, spy, sry);
            Rv = T{srx, sry};
            // hf = (y_{n+1} + y_n) / 2 with the halving on the integer pipe
            const double Px = fma(h48, spx, half_exp(xv.x + y0v.x)), Py = fma(h48, spy, half_exp(xv.y + y0v.y));
            qv = make_double2(fma(-c161h, srx, Px), fma(-c161h, sry, Py));
            mv = T{fma(-c161h, pcv.x, Px), fma(-c161h, pcv.y, Py)};
          } else {
            const T Y = T{y0c * f.x + y1c * e0.x + y2c * e1.x + y3c * e2.x, y0c * f.y + y1c * e0.y + y2c * e1.y + y3c * e2.y};
            Rv = T{r0c * f.x + r1c * e0.x + r2c * e1.x + r3c * e2.x, r0c * f.y + r1c * e0.y + r2c * e1.y + r3c * e2.y};
            const double2 Yd = to_d(Y);
            qv = make_double2(fma(0.5, xv.x, fma(0.5, y0v.x, Yd.x)), fma(0.5, xv.y, fma(0.5, y0v.y, Yd.y)));
            mv = to_r<R>(make_double2(fma((double)c161, (double)(Rv.x - pcv.x), qv.x),
                                      fma((double)c161, (double)(Rv.y - pcv.y), qv.y)));
          }
          reinterpret_cast<T*>(a.m)[i] = mv;
          a.q[i] = qv;
          reinterpret_cast<T*>(a.r)[i] = Rv;
          mo[c] = mv;
        }
        if constexpr (sizeof(R) == 4)
          dens_acc(mo[0], mo[1], dF);
        else
          dens_acc(mo[0], mo[1], sn, sr, si);
      }
    }
    if constexpr (MODE == M_ETA) {
      // deterministic block sums (any block size): every thread stores its value,
      // thread j adds the NT values of state j in thread order
      __shared__ double red[QB][NT];
#pragma unroll
      for (int j = 0; j < QB; ++j) red[j][threadIdx.x] = eta_acc[j];
      __syncthreads();
      if ((int)threadIdx.x < QB && qb0 + (int)threadIdx.x < q_end) {
        double t = 0.0;
        for (int k = 0; k < NT; ++k) t += red[threadIdx.x][k];
        a.eta_part[(long)(qb0 + threadIdx.x) * nbx + bx] = t;
      }
    }
    // the batch buffer is reused
    if constexpr (kPrefetch) {
      if (__syncthreads_or(failed)) break;
    } else {
      __syncthreads();
    }
  }
  if constexpr (kPrefetch) {
    // a block that stopped early lets the copies it issued land before it exits
    if (threadIdx.x == 0) {
      if (pend[0]) um::mbar_wait(&mb_stage[0], ph_x, kDrainPolls);
      if (pend[1]) um::mbar_wait(&mb_stage[1], ph_q, kDrainPolls);
    }
  }
  if (a.dens) {
    if constexpr (sizeof(R) == 4) dens_fold(dF, sn, sr, si);
    const long o = (long)g * nxyz + site;
    a.part_n[o] = 2.0 * sn;
    if (MODE != M_ENERGY) {
      a.part_nr[o] = sr;
      a.part_ni[o] = si;
    }
  }
}

#define LISE_PENCILS_BOUNDS                                                                                    \
  __launch_bounds__(N * TX, (N * TX >= 384 && sizeof(R) == 4) || N * TX == 256                                 \
                                ? 2                                                                            \
                                : ((sizeof(R) == 8 && N * TX == 128) ? 7 : ((sizeof(R) == 8 && N * TX == 192) ? 3 : 1)))

template <typename R, int N, int TX, int QB, int MODE, bool ST = false>
__global__ void LISE_PENCILS_BOUNDS k_pencils(const __grid_constant__ PencilArgs a) {
  pencils_body<R, N, TX, QB, MODE, ST>(a, blockIdx.y, blockIdx.x, gridDim.x);
}

// Several evolutions of one lattice size in one launch: block row blockIdx.y is the item
// (evolution, group) b.items[blockIdx.y], with that evolution's arguments b.evo[evolution]
// (device memory, tensor maps included).
template <typename R, int N, int TX, int QB, int MODE, bool ST = false>
__global__ void LISE_PENCILS_BOUNDS k_pencils_batch(const __grid_constant__ PencilBatch b) {
  const int2 it = b.items[blockIdx.y];
  pencils_body<R, N, TX, QB, MODE, ST>(b.evo[it.x], it.y, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------- reduce/potentials --
__device__ __forceinline__ void neumaier(double& s, double& c, double x) {
  double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

__device__ __forceinline__ void reduce_body(const ReduceArgs& a, const long s) {
  if (s >= a.nxyz) return;
  double n = 0, cn = 0, r = 0, cr = 0, i = 0, ci = 0;
  for (int g = 0; g < a.n_groups; ++g) {
    const long o = (long)g * a.nxyz + s;
    neumaier(n, cn, a.part_n[o]);
    neumaier(r, cr, a.part_nr[o]);
    neumaier(i, ci, a.part_ni[o]);
  }
  n += cn;
  r += cr;
  i += ci;
  if (a.avg_n) {
    n = 0.5 * (n + a.avg_n[s]);
    const double2 o = a.avg_nu[s];
    r = 0.5 * (r + o.x);
    i = 0.5 * (i + o.y);
  }
  if (!(isfinite(n) && isfinite(r) && isfinite(i))) atomicOr(a.err, 1);
  a.n_out[s] = n;
  a.nu_out[s] = make_double2(r, i);
  if (!a.W) return;
  const double PI = 3.14159265358979323846;
  const double cb = cbrt(3.0 * PI * PI * n);
  const int iz = (int)(s / ((long)a.N * a.N));
  double v = a.v_static ? a.v_static[s] : 0.0;
  v += (a.drive_ptr ? *a.drive_ptr : a.drive) * ((iz - a.N / 2) * a.a);
  const double U = 0.5 * a.beta * cb * cb;
  double geff, dgeff;
  pairing_geff(a.pair, n, cb * cb, U + v, &geff, &dgeff);
  a.W[s] = U + dgeff * (r * r + i * i) - a.mu + v;  // U(n) + dE_pair/dn - mu + V_ext
  a.D[s] = make_double2(-geff * r, -geff * i);                            // Delta = -g_eff nu
}

__global__ void k_reduce(ReduceArgs a) { reduce_body(a, (long)blockIdx.x * blockDim.x + threadIdx.x); }

// Several evolutions in one launch: evolution k owns blocks [b.block0[k], b.block0[k + 1]).
__global__ void k_reduce_batch(ReduceBatch b) {
  int k = 0;
  while (k + 1 < b.n && (long)blockIdx.x >= b.block0[k + 1]) ++k;
  reduce_body(b.evo[k], ((long)blockIdx.x - b.block0[k]) * blockDim.x + threadIdx.x);
}

// --------------------------------------------------------------- pointwise --
// Eq. p, Eq. m and the corrector's Q, R (see lise_kernels.cuh) from the history
//   y0 = y_{k}, y1 = y_{k-1}, d0..d3 = y'_{k}..y'_{k-3}, pc = p_k - c_k,
// plus the densities of m.  Used after the start procedure (k = 3) and, in the
// mixed path, as the second half of every derivative/predictor step.  As in the
// fused epilogue, the derivative combinations run in the compute precision R and
// every sum with a state value in FP64.
//
// ST (FP32 compute precision): the strict split of LISE_MIXED_STRICT.  The derivative sums
// are taken exactly in integers from the FP32 derivatives (pred_sums on their exact FP64
// values: sp = 48 pt / h, sr = 48 R / h, each rounded once), R and p - c are complex128 in
// units of h/48 (as in the FP64 path), P = hf + pt, Q = P - (161/170) R and
// m = P - (161/170)(p - c) in FP64; m is rounded to FP32 only as the operand of the next
// FP32 H psi, and its densities are taken from its FP64 value.
template <typename R, bool ST>
__device__ __forceinline__ void predict_body(const PointwiseArgs& a, const long s, const int g) {
  using T = typename Cx<R>::T;
  if (s >= a.nxyz) return;
  const int q_begin = g * a.qg, q_end = min(a.n_qp, q_begin + a.qg);
  const R h48 = (R)(a.h / 48.0);
  const R c161 = (R)(161.0 / 170.0), c9 = (R)(9.0 / 170.0);
  double sn = 0, sr = 0, si = 0;
  DensF dF;  // FP32 operands (mixed path)
  if constexpr (ST) {
    const double h48d = a.h / 48.0, c161h = 161.0 / 170.0 * h48d;
    for (int q = q_begin; q < q_end; ++q) {
      double2 md[2];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const long i = (long)(2 * q + c) * a.nxyz + s;
        const double2 e0 = to_d(reinterpret_cast<const T*>(a.d0)[i]), e1 = to_d(reinterpret_cast<const T*>(a.d1)[i]),
                      e2 = to_d(reinterpret_cast<const T*>(a.d2)[i]), e3 = to_d(reinterpret_cast<const T*>(a.d3)[i]);
        double spx, srx, spy, sry;
        pred_sums(e0.x, e1.x, e2.x, e3.x, spx, srx);
        pred_sums(e0.y, e1.y, e2.y, e3.y, spy, sry);
        const double2 pcv = reinterpret_cast<const double2*>(a.pc)[i];
        const double2 y0 = a.y0[i], y1 = a.y1[i];
        const double Px = fma(h48d, spx, half_exp(y0.x + y1.x)), Py = fma(h48d, spy, half_exp(y0.y + y1.y));
        a.q[i] = make_double2(fma(-c161h, srx, Px), fma(-c161h, sry, Py));
        reinterpret_cast<double2*>(a.r)[i] = make_double2(srx, sry);
        md[c] = make_double2(fma(-c161h, pcv.x, Px), fma(-c161h, pcv.y, Py));
        reinterpret_cast<T*>(a.m)[i] = to_r<R>(md[c]);
      }
      dens_acc(md[0], md[1], sn, sr, si);
    }
  } else {
    for (int q = q_begin; q < q_end; ++q) {
      T mo[2];  // m in the compute precision, for its densities
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const long i = (long)(2 * q + c) * a.nxyz + s;
        const T e0 = reinterpret_cast<const T*>(a.d0)[i], e1 = reinterpret_cast<const T*>(a.d1)[i],
                e2 = reinterpret_cast<const T*>(a.d2)[i], e3 = reinterpret_cast<const T*>(a.d3)[i];
        const T pcv = reinterpret_cast<const T*>(a.pc)[i];
        const T pt = T{h48 * (R(119) * e0.x - R(99) * e1.x + R(69) * e2.x - R(17) * e3.x),
                       h48 * (R(119) * e0.y - R(99) * e1.y + R(69) * e2.y - R(17) * e3.y)};
        const T ct = T{h48 * (R(51) * e0.x + R(3) * e1.x + e2.x), h48 * (R(51) * e0.y + R(3) * e1.y + e2.y)};
        // FP64 keeps p - c and R in units of h/48 (as the FP64 pencils epilogues do)
        const R cpc = sizeof(R) == 8 ? c161 * h48 : c161;
        const T X = T{pt.x - cpc * pcv.x, pt.y - cpc * pcv.y};
        const T Y = T{c161 * ct.x + c9 * pt.x, c161 * ct.y + c9 * pt.y};
        const double2 y0 = a.y0[i], y1 = a.y1[i];
        if constexpr (sizeof(R) == 4) {
          // Q = (y0 + y1)/2 + Y in FP64 (two FMAs); m = Q + (X - Y) only needs FP32,
          // the precision it is stored and used in
          const double2 Yd = to_d(Y);
          const double2 qv = make_double2(fma(0.5, y0.x, fma(0.5, y1.x, Yd.x)), fma(0.5, y0.y, fma(0.5, y1.y, Yd.y)));
          a.q[i] = qv;
          const T qr = to_r<R>(qv);
          const T mr = T{qr.x + (X.x - Y.x), qr.y + (X.y - Y.y)};
          reinterpret_cast<T*>(a.m)[i] = mr;
          mo[c] = mr;
        } else {
          const double2 hf = dscale(dadd(y0, y1), 0.5);
          const double2 mv = dadd(hf, to_d(X));
          reinterpret_cast<T*>(a.m)[i] = to_r<R>(mv);
          a.q[i] = dadd(hf, to_d(Y));
          mo[c] = to_r<R>(mv);
        }
        if constexpr (sizeof(R) == 8)
          reinterpret_cast<T*>(a.r)[i] = T{R(68) * e0.x - R(102) * e1.x + R(68) * e2.x - R(17) * e3.x,
                                           R(68) * e0.y - R(102) * e1.y + R(68) * e2.y - R(17) * e3.y};
        else
          reinterpret_cast<T*>(a.r)[i] = T{pt.x - ct.x, pt.y - ct.y};
      }
      if constexpr (sizeof(R) == 4)
        dens_acc(mo[0], mo[1], dF);
      else
        dens_acc(mo[0], mo[1], sn, sr, si);
    }
    if constexpr (sizeof(R) == 4) dens_fold(dF, sn, sr, si);
  }
  const long o = (long)g * a.nxyz + s;
  a.part_n[o] = 2.0 * sn;
  a.part_nr[o] = sr;
  a.part_ni[o] = si;
}

template <typename R, bool ST = false>
__global__ void k_predict(PointwiseArgs a) {
  predict_body<R, ST>(a, (long)blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y);
}

// Several evolutions of one lattice size in one launch: block row blockIdx.y is the item
// (evolution, group) b.items[blockIdx.y].
template <typename R, bool ST = false>
__global__ void k_predict_batch(PredictBatch b) {
  const int2 it = b.items[blockIdx.y];
  predict_body<R, ST>(b.evo[it.x], (long)blockIdx.x * blockDim.x + threadIdx.x, it.y);
}

__global__ void k_density(PointwiseArgs a) {
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nxyz) return;
  const int g = blockIdx.y;
  const int q_begin = g * a.qg, q_end = min(a.n_qp, q_begin + a.qg);
  double sn = 0, sr = 0, si = 0;
  for (int q = q_begin; q < q_end; ++q) {
    const long i = (long)(2 * q) * a.nxyz + s;
    dens_acc(a.src[i], a.src[i + a.nxyz], sn, sr, si);
  }
  const long o = (long)g * a.nxyz + s;
  a.part_n[o] = 2.0 * sn;
  a.part_nr[o] = sr;
  a.part_ni[o] = si;
}

// Energy density per site (times a^3) and a^3 n, for the host's final sum.
// E = a^3 sum_r [(alpha/2) tau + (3/10) beta (3 pi^2)^(2/3) n^(5/3) + g |nu|^2 + V n]
// (Eq. pairing has + g_eff |kappa|^2); part holds sum_k 2 Re(v_k^* T v_k).
__global__ void k_energy_sites(const double* part, int n_groups, const double* nd, const double2* nu,
                               const double* v_static, double drive, Pairing pair, int N, double a, double* out) {
  const long nxyz = (long)N * N * N;
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nxyz) return;
  double ek = 0, ck = 0;
  for (int k = 0; k < n_groups; ++k) neumaier(ek, ck, part[(long)k * nxyz + s]);
  ek += ck;
  const double PI = 3.14159265358979323846;
  const double n = nd[s];
  const double cb = cbrt(3.0 * PI * PI);
  const double cn = cbrt(n);
  const int iz = (int)(s / ((long)N * N));
  double v = v_static ? v_static[s] : 0.0;
  v += drive * ((iz - N / 2) * a);
  const double2 w = nu[s];
  const double a3 = a * a * a;
  const double cb2 = cb * cb * cn * cn;  // (3 pi^2 n)^(2/3)
  double geff, dgeff;
  pairing_geff(pair, n, cb2, 0.5 * pair.beta * cb2 + v, &geff, &dgeff);
  out[s] = a3 * (ek + 0.3 * pair.beta * cb * cb * n * cn * cn + geff * (w.x * w.x + w.y * w.y) + v * n);
  out[nxyz + s] = a3 * n;
}

__global__ void k_eta_reduce(const double* part, int n_qp, int n_blocks, double a3, double* eta) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_qp) return;
  double s = 0, c = 0;
  for (int b = 0; b < n_blocks; ++b) neumaier(s, c, part[(long)q * n_blocks + b]);
  eta[q] = a3 * (s + c);
}

// Current density partials (Eq. j): one block per x-line (y, z), one thread per x, one grid
// row per state group; d/dx from the line in shared memory, d/dy and d/dz from global
// (coalesced across the block).  Dense circulant sums in FP64: an observable, not the step.
__global__ void k_currents(const double2* psi, const double* d1g, int N, int n_qp, int qg, double* jx, double* jy,
                           double* jz) {
  extern __shared__ double2 cur_smem[];
  double2* line = cur_smem;                               // [N]
  double* d1 = reinterpret_cast<double*>(line + N);       // [N]
  const int x = threadIdx.x;
  const int y = blockIdx.x % N, z = blockIdx.x / N;
  const long nxyz = (long)N * N * N;
  const long site = ((long)z * N + y) * N + x;
  for (int i = x; i < N; i += blockDim.x) d1[i] = d1g[i];
  const int g = blockIdx.y;
  const int q0 = g * qg, q1 = min(n_qp, q0 + qg);
  double sx = 0, sy = 0, sz = 0;
  for (int q = q0; q < q1; ++q) {
    const double2* v = psi + ((long)q * 2 + 1) * nxyz;  // v component of state q
    __syncthreads();
    line[x] = v[site];
    __syncthreads();
    const double2 vv = line[x];
    double2 dx = make_double2(0, 0), dy = make_double2(0, 0), dz = make_double2(0, 0);
    for (int k = 0; k < N; ++k) {
      const double wx = d1[(x - k + N) % N], wy = d1[(y - k + N) % N], wz = d1[(z - k + N) % N];
      const double2 ax = line[k];
      const double2 ay = v[((long)z * N + k) * N + x];
      const double2 az = v[((long)k * N + y) * N + x];
      dx.x = fma(wx, ax.x, dx.x); dx.y = fma(wx, ax.y, dx.y);
      dy.x = fma(wy, ay.x, dy.x); dy.y = fma(wy, ay.y, dy.y);
      dz.x = fma(wz, az.x, dz.x); dz.y = fma(wz, az.y, dz.y);
    }
    // -2 Im(conj(v) d) = -2 (v.x d.y - v.y d.x)
    sx -= 2.0 * (vv.x * dx.y - vv.y * dx.x);
    sy -= 2.0 * (vv.x * dy.y - vv.y * dy.x);
    sz -= 2.0 * (vv.x * dz.y - vv.y * dz.x);
  }
  const long o = (long)g * nxyz + site;
  jx[o] = sx;
  jy[o] = sy;
  jz[o] = sz;
}

__global__ void k_sum_groups3(const double* jx, const double* jy, const double* jz, int n_groups, long nxyz,
                              double* out) {
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= nxyz) return;
  double a = 0, b = 0, c = 0;
  for (int g = 0; g < n_groups; ++g) {
    a += jx[(long)g * nxyz + s];
    b += jy[(long)g * nxyz + s];
    c += jz[(long)g * nxyz + s];
  }
  out[s] = a;
  out[nxyz + s] = b;
  out[2 * nxyz + s] = c;
}

// Norm partials: block b of state q sums |x|^2 over its slice of the state's 2 nxyz
// elements (strided per thread, then a fixed-order tree in shared memory).
__global__ void k_norm_part(const double2* y, long nxyz, int nb, double* part) {
  __shared__ double red[256];
  const int q = blockIdx.y, b = blockIdx.x;
  const long n = 2 * nxyz, chunk = (n + nb - 1) / nb;
  const long i0 = (long)b * chunk, i1 = min(n, i0 + chunk);
  const double2* x = y + (long)q * n;
  double s = 0.0;
  for (long i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, s));
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[(long)q * nb + b] = red[0];
}

__global__ void k_norm_scale(const double* part, int n_qp, int nb, double a3, double* scale) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_qp) return;
  double s = 0, c = 0;
  for (int b = 0; b < nb; ++b) neumaier(s, c, part[(long)q * nb + b]);
  scale[q] = 1.0 / sqrt(a3 * (s + c));
}

// y *= scale per state (in place) and the density partials of the scaled state.
__global__ void k_scale_density(double2* y, const double* scale, PointwiseArgs a) {
  const long s = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= a.nxyz) return;
  const int g = blockIdx.y;
  const int q_begin = g * a.qg, q_end = min(a.n_qp, q_begin + a.qg);
  double sn = 0, sr = 0, si = 0;
  for (int q = q_begin; q < q_end; ++q) {
    const long i = (long)(2 * q) * a.nxyz + s;
    const double f = scale[q];
    const double2 u = dscale(y[i], f), v = dscale(y[i + a.nxyz], f);
    y[i] = u;
    y[i + a.nxyz] = v;
    dens_acc(u, v, sn, sr, si);
  }
  const long o = (long)g * a.nxyz + s;
  a.part_n[o] = 2.0 * sn;
  a.part_nr[o] = sr;
  a.part_ni[o] = si;
}

// Eq. kick: u -> e^{i chi} u, v -> e^{-i chi} v.
__global__ void k_kick(const double2* src, double2* dst, const double* chi, long count, long nxyz) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const long site = i % nxyz;
    const bool v = (i / nxyz) & 1;  // component index within the state
    double sn, cs;
    sincos(chi[site], &sn, &cs);
    if (v) sn = -sn;
    const double2 x = src[i];
    dst[i] = make_double2(x.x * cs - x.y * sn, x.x * sn + x.y * cs);
  }
}

__global__ void k_finite(const double2* x, long count, int* err) {
  int bad = 0;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long)gridDim.x * blockDim.x) {
    const double2 v = x[i];
    if (!(isfinite(v.x) && isfinite(v.y))) bad = 1;
  }
  if (bad) atomicOr(err, 2);
}

// ---------------------------------------------------------------- launchers --
// cudaFuncSetAttribute acts on the current device only: raise a kernel's dynamic shared
// memory limit once on every device it is launched on (done: one bit per device ordinal).
static int smem_attr(const void* kern, size_t bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 3;
  const unsigned long long bit = dev >= 0 && dev < 64 ? (1ull << dev) : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes) != cudaSuccess) return 3;
  if (bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return 0;
}

bool supported_n(int N) {
  switch (N) {
    case 8: case 12: case 16: case 20: case 24: case 32: case 40: case 48: case 64: return true;
    default: return false;
  }
}
int pencil_tx(int N, int mixed) { return (ozaki_path(N, mixed) || N % 8 != 0) ? 4 : 8; }
int pencil_qb(int N, int mixed) {
  const int t = pencil_qb_get(N, mixed);
  return t ? t : ((N >= 40 || (N >= 32 && (mixed || ozaki_path(N, mixed)))) ? 2 : 4);
}

template <int N>
static int planes_oz_n(const PlanesArgs& a, cudaStream_t s) {
  using P = OzPlanes<N>;
  auto kern = k_planes_oz<N>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, P::smem, attr_done)) return 3;
  const long blocks = (a.n_planes + P::PB - 1) / P::PB;
  if (blocks <= 0) return 0;
  if (!a.ozb) return 1;
  kern<<<(unsigned)blocks, 256, P::smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// persistent: one warp-specialised block per SM (48-point lines, chunked tensor memory)
template <int N>
static int planes_tcc_n(const PlanesArgs& a, cudaStream_t s) {
  using P = TcPlanesC<N>;
  auto kern = k_planes_tcc<N>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, P::smem, attr_done)) return 3;
  if (a.n_planes <= 0) return 0;
  if (!a.ozb) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 3;
  const long blocks = std::min<long>(a.n_planes, (long)sms);
  kern<<<(unsigned)blocks, kTccThreads, P::smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// persistent: one warp-specialised block per SM, each walking the planes
template <int N>
static int planes_tc_n(const PlanesArgs& a, cudaStream_t s) {
  using P = TcPlanes<N>;
  auto kern = k_planes_tc<N>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, P::smem, attr_done)) return 3;
  if (a.n_planes <= 0) return 0;
  if (!a.ozb) return 1;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 3;
  const long blocks = std::min<long>(a.n_planes, (long)sms);
  kern<<<(unsigned)blocks, kWsThreads, P::smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// Planes per block of the FFT planes kernel: the variants compiled for a lattice (shared
// memory within 227 KB, at most 32 values per thread in registers); the default is
// PlanesPB<N>, a tuned value replaces it (lise_api.cu: tune_planes).  Every plane is
// transformed on its own, so the choice does not change any result.
template <typename R, int N, int PB>
constexpr bool planes_pb_fits() {
  using T = typename Cx<R>::T;
  return (size_t)PB * N * (N + 1) * sizeof(T) + N * sizeof(T) + N * sizeof(R) <= 227 * 1024 &&
         (PB * N * N + 255) / 256 <= 32;
}
static std::atomic<int> g_pb_tuned[2][65];  // 0: not tuned

int planes_pb_get(int N, int mixed) {
  if (N < 0 || N > 64) return 0;
  return g_pb_tuned[mixed ? 1 : 0][N].load(std::memory_order_relaxed);
}
void planes_pb_set(int N, int mixed, int pb) {
  if (N >= 0 && N <= 64) g_pb_tuned[mixed ? 1 : 0][N].store(pb, std::memory_order_relaxed);
}

// The register-line variants (planes_line_body, planes_half_body), FP32 compute precision only:
// LineTpl threads per line, whole warps of lines for the two-thread form, shared memory within
// 227 KB.
template <typename R, int N, int PB>
constexpr bool planes_line_fits() {
  return sizeof(R) == 4 && LineTpl<N>::v * PB * N <= 1024 && (LineTpl<N>::v == 1 || PB * N % 16 == 0) &&
         (size_t)PB * N * (N + 1) * sizeof(float2) + N * sizeof(float2) + N * sizeof(float) <= 227 * 1024;
}
template <int N, int PB>
constexpr size_t planes_line_smem() {
  return (size_t)PB * N * (N + 1) * sizeof(float2) + N * sizeof(float2) + N * sizeof(float);
}

template <int N, int PB>
static int planes_line_npb(const PlanesArgs& a, cudaStream_t s) {
  auto kern = k_planes_line<N, PB>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, planes_line_smem<N, PB>(), attr_done)) return 3;
  const long blocks = (a.n_planes + PB - 1) / PB;
  if (blocks <= 0) return 0;
  kern<<<(unsigned)blocks, LineTpl<N>::v * PB * N, planes_line_smem<N, PB>(), s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

template <typename R, int N, int PB>
static int planes_npb(const PlanesArgs& a, cudaStream_t s) {
  using T = typename Cx<R>::T;
  constexpr int NT = 256;
  const size_t smem = (size_t)PB * N * (N + 1) * sizeof(T) + N * sizeof(T) + N * sizeof(R);
  auto kern = k_planes<R, N, PB, NT>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, smem, attr_done)) return 3;
  const long blocks = (a.n_planes + PB - 1) / PB;
  if (blocks <= 0) return 0;
  kern<<<(unsigned)blocks, NT, smem, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

template <typename R, int N>
static int planes_n(const PlanesArgs& a, cudaStream_t s, int pb) {
  if constexpr (pencil_oz<R, N>()) {
    if constexpr (N == 32)
      return planes_tc_n<N>(a, s);
    else if constexpr (N == 48)
      return planes_tcc_n<N>(a, s);
    else
      return planes_oz_n<N>(a, s);
  } else {
    if (pb == 0) pb = planes_pb_get(N, sizeof(R) == 4);
    if constexpr (planes_line_fits<R, N, 1>())
      if (pb == -1) return planes_line_npb<N, 1>(a, s);
    if constexpr (planes_line_fits<R, N, 2>())
      if (pb == -2) return planes_line_npb<N, 2>(a, s);
    if constexpr (planes_line_fits<R, N, 4>())
      if (pb == -4) return planes_line_npb<N, 4>(a, s);
    if constexpr (planes_line_fits<R, N, 8>())
      if (pb == -8) return planes_line_npb<N, 8>(a, s);
    if constexpr (planes_pb_fits<R, N, 1>())
      if (pb == 1) return planes_npb<R, N, 1>(a, s);
    if constexpr (planes_pb_fits<R, N, 2>())
      if (pb == 2) return planes_npb<R, N, 2>(a, s);
    if constexpr (planes_pb_fits<R, N, 4>())
      if (pb == 4) return planes_npb<R, N, 4>(a, s);
    if constexpr (planes_pb_fits<R, N, 8>())
      if (pb == 8) return planes_npb<R, N, 8>(a, s);
    return planes_npb<R, N, PlanesPB<N>::v>(a, s);
  }
}

template <typename R, int N>
static bool planes_pb_valid_n(int pb) {
  if constexpr (pencil_oz<R, N>()) {
    return false;
  } else {
    switch (pb) {
      case 1: return planes_pb_fits<R, N, 1>();
      case 2: return planes_pb_fits<R, N, 2>();
      case 4: return planes_pb_fits<R, N, 4>();
      case 8: return planes_pb_fits<R, N, 8>();
      case -1: return planes_line_fits<R, N, 1>();
      case -2: return planes_line_fits<R, N, 2>();
      case -4: return planes_line_fits<R, N, 4>();
      case -8: return planes_line_fits<R, N, 8>();
      default: return false;
    }
  }
}

// ----------------------------------------------------- pencil batch autotune --
// States per batch (QB) of the pencils kernel: a default per lattice and precision, or
// the value an autotuning pass measured fastest (lise_api.cu: tune_pencils).  QB only
// changes how a block walks its states (the per-thread density sums and every per-state
// operation keep their order), so results are bitwise identical for every QB.
template <typename R, int N>
constexpr int qb_default() {
  // fewer states per batch at large N (registers), for the FP32 path from N = 32 (staging)
  // and for the FP64 tensor-core path from N = 32 (registers for four resident blocks)
  return (N >= 40 || (sizeof(R) == 4 && N >= 32) || (pencil_oz<R, N>() && N >= 32)) ? 2 : 4;
}
template <typename R, int N, int QB>
constexpr bool qb_fits() {
  using T = typename Cx<R>::T;
  constexpr int TX = pencil_tx_c<R, N>();
  return pencil_smem_bytes<T, N, TX, QB>() <= 227 * 1024;
}

static std::atomic<int> g_qb_tuned[2][65];  // 0: not tuned

int pencil_qb_get(int N, int mixed) {
  if (N < 0 || N > 64) return 0;
  return g_qb_tuned[mixed ? 1 : 0][N].load(std::memory_order_relaxed);
}
void pencil_qb_set(int N, int mixed, int qb) {
  if (N >= 0 && N <= 64) g_qb_tuned[mixed ? 1 : 0][N].store(qb, std::memory_order_relaxed);
}

// Tensor map of a state-shaped array [2 n_qp planes][N z][N y][N x] of complex values
// (complex64, or complex128 when c128) for the pencils kernel's staging boxes
// [2 QB planes][N z][1 y][TX x]; the innermost dimension counts real words.
static bool encode_stage_map(CUtensorMap* m, const void* base, bool c128, int N, int n_qp, int TX, int QB) {
  using Fn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*, const cuuint64_t*,
                          const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                          CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static const Fn encode = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      return (Fn) nullptr;
    return reinterpret_cast<Fn>(f);
  }();
  if (!encode || !base) return false;
  const cuuint64_t w = c128 ? 8 : 4;
  const cuuint64_t dims[4] = {(cuuint64_t)2 * N, (cuuint64_t)N, (cuuint64_t)N, (cuuint64_t)2 * n_qp};
  const cuuint64_t strides[3] = {2 * N * w, 2 * (cuuint64_t)N * N * w, 2 * (cuuint64_t)N * N * N * w};
  const cuuint32_t box[4] = {(cuuint32_t)(2 * TX), 1, (cuuint32_t)N, (cuuint32_t)(2 * QB)};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return encode(m, c128 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<void*>(base),
                dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <typename R, int N, int MODE, int QB, bool ST>
static int pencils_nmq(const PencilArgs& a, cudaStream_t s) {
  using T = typename Cx<R>::T;
  constexpr int TX = pencil_tx_c<R, N>();
  const size_t smem = (size_t)pencil_smem_bytes<T, N, TX, QB>();
  auto kern = k_pencils<R, N, TX, QB, MODE, ST>;
  if (pencil_oz<R, N>() && !a.ozb) return 1;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, smem, attr_done)) return 3;
  const int n_groups = (a.n_qp + a.qg - 1) / a.qg;
  dim3 grid((N / TX) * N, n_groups);
  if constexpr (sizeof(R) == 4) {
    // the staged arrays of the FP32 compute precision: tensor maps for this launch
    PencilArgs b = a;
    const bool ok = encode_stage_map(&b.tm_x, a.xr ? a.xr : (const void*)a.x, !a.xr, N, a.n_qp, TX, QB) &&
                    encode_stage_map(&b.tm_t, a.txy, false, N, a.n_qp, TX, QB) &&
                    (MODE != M_CORRECT || (encode_stage_map(&b.tm_q, a.q, true, N, a.n_qp, TX, QB) &&
                                           (ST || encode_stage_map(&b.tm_r, a.r, false, N, a.n_qp, TX, QB))));
    if (!ok) return 3;
    kern<<<grid, N * TX, smem, s>>>(b);
  } else {
    kern<<<grid, N * TX, smem, s>>>(a);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

// the strict-split corrector (LISE_MIXED_STRICT) of the FP32 compute precision, else the plain one
template <typename R, int N, int MODE, int QB>
static int pencils_nmq_st(const PencilArgs& a, cudaStream_t s) {
  if constexpr (sizeof(R) == 4 && MODE == M_CORRECT)
    if (a.strict) return pencils_nmq<R, N, MODE, QB, true>(a, s);
  return pencils_nmq<R, N, MODE, QB, false>(a, s);
}

// the step's modes have QB = 2 and QB = 4 variants (where they fit); the others use the default
template <typename R, int N, int MODE>
static int pencils_nm(const PencilArgs& a, cudaStream_t s, int qb) {
  constexpr bool kTunable = MODE == M_RHS || MODE == M_CORRECT || MODE == M_DERIV_PREDICT;
  if constexpr (kTunable) {
    if (qb == 0) qb = pencil_qb_get(N, sizeof(R) == 4);
    if constexpr (pencil_oz<R, N>())
      if (qb == 1) return pencils_nmq_st<R, N, MODE, 1>(a, s);
    if constexpr (qb_fits<R, N, 2>())
      if (qb == 2) return pencils_nmq_st<R, N, MODE, 2>(a, s);
    if constexpr (qb_fits<R, N, 4>())
      if (qb == 4) return pencils_nmq_st<R, N, MODE, 4>(a, s);
  }
  return pencils_nmq_st<R, N, MODE, qb_default<R, N>()>(a, s);
}

#define LISE_FOR_N(X) X(8) X(12) X(16) X(20) X(24) X(32) X(40) X(48) X(64)

// ------------------------------------------------------------- batched launches --
// The FP32 compute precision (the batched path serves the mixed splits).
template <int N, int MODE, int QB, bool ST>
static int pencils_batch_nmq(const PencilBatch& b, int n_items, cudaStream_t s) {
  using T = float2;
  constexpr int TX = pencil_tx_c<float, N>();
  const size_t smem = (size_t)pencil_smem_bytes<T, N, TX, QB>();
  auto kern = k_pencils_batch<float, N, TX, QB, MODE, ST>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, smem, attr_done)) return 3;
  if (n_items <= 0) return 0;
  kern<<<dim3((N / TX) * N, n_items), N * TX, smem, s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

template <int N, int MODE, bool ST>
static int pencils_batch_nm(const PencilBatch& b, int n_items, int qb, cudaStream_t s) {
  if constexpr (qb_fits<float, N, 2>())
    if (qb == 2) return pencils_batch_nmq<N, MODE, 2, ST>(b, n_items, s);
  if constexpr (qb_fits<float, N, 4>())
    if (qb == 4) return pencils_batch_nmq<N, MODE, 4, ST>(b, n_items, s);
  return 1;
}

template <int N>
static int pencils_batch_n(int mode, int strict, const PencilBatch& b, int n_items, int qb, cudaStream_t s) {
  if (mode == M_CORRECT)
    return strict ? pencils_batch_nm<N, M_CORRECT, true>(b, n_items, qb, s)
                  : pencils_batch_nm<N, M_CORRECT, false>(b, n_items, qb, s);
  if (mode == M_RHS) return pencils_batch_nm<N, M_RHS, false>(b, n_items, qb, s);
  return 1;
}

template <int N, int PB>
static int planes_batch_npb(const PlanesBatch& b, long n_blocks, cudaStream_t s) {
  constexpr int NT = 256;
  const size_t smem = (size_t)PB * N * (N + 1) * sizeof(float2) + N * sizeof(float2) + N * sizeof(float);
  auto kern = k_planes_batch<float, N, PB, NT>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, smem, attr_done)) return 3;
  if (n_blocks <= 0) return 0;
  kern<<<(unsigned)n_blocks, NT, smem, s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

template <int N, int PB>
static int planes_line_batch_npb(const PlanesBatch& b, long n_blocks, cudaStream_t s) {
  auto kern = k_planes_line_batch<N, PB>;
  static std::atomic<unsigned long long> attr_done{0};
  if (smem_attr((const void*)kern, planes_line_smem<N, PB>(), attr_done)) return 3;
  if (n_blocks <= 0) return 0;
  kern<<<(unsigned)n_blocks, LineTpl<N>::v * PB * N, planes_line_smem<N, PB>(), s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

template <int N>
static int planes_batch_n(const PlanesBatch& b, long n_blocks, int pb, cudaStream_t s) {
  if constexpr (planes_line_fits<float, N, 1>())
    if (pb == -1) return planes_line_batch_npb<N, 1>(b, n_blocks, s);
  if constexpr (planes_line_fits<float, N, 2>())
    if (pb == -2) return planes_line_batch_npb<N, 2>(b, n_blocks, s);
  if constexpr (planes_line_fits<float, N, 4>())
    if (pb == -4) return planes_line_batch_npb<N, 4>(b, n_blocks, s);
  if constexpr (planes_line_fits<float, N, 8>())
    if (pb == -8) return planes_line_batch_npb<N, 8>(b, n_blocks, s);
  if constexpr (planes_pb_fits<float, N, 1>())
    if (pb == 1) return planes_batch_npb<N, 1>(b, n_blocks, s);
  if constexpr (planes_pb_fits<float, N, 2>())
    if (pb == 2) return planes_batch_npb<N, 2>(b, n_blocks, s);
  if constexpr (planes_pb_fits<float, N, 4>())
    if (pb == 4) return planes_batch_npb<N, 4>(b, n_blocks, s);
  if constexpr (planes_pb_fits<float, N, 8>())
    if (pb == 8) return planes_batch_npb<N, 8>(b, n_blocks, s);
  return 1;
}

int launch_pencils_batch(int N, int mode, int strict, const PencilBatch& b, int n_items, int qb, cudaStream_t s) {
  switch (N) {
#define CASE(n) \
  case n: return pencils_batch_n<n>(mode, strict, b, n_items, qb, s);
    LISE_FOR_N(CASE)
#undef CASE
    default: return 1;
  }
}

int launch_planes_batch(int N, int pb, const PlanesBatch& b, long n_blocks, cudaStream_t s) {
  switch (N) {
#define CASE(n) \
  case n: return planes_batch_n<n>(b, n_blocks, pb, s);
    LISE_FOR_N(CASE)
#undef CASE
    default: return 1;
  }
}

long planes_blocks(long n_planes, int pb) {
  const int p = pb < 0 ? -pb : pb;  // (negative: the register-line variant with -pb planes per block)
  return p > 0 ? (n_planes + p - 1) / p : 0;
}

int launch_reduce_batch(const ReduceBatch& b, long n_blocks, cudaStream_t s) {
  if (n_blocks <= 0) return 0;
  k_reduce_batch<<<(unsigned)n_blocks, 256, 0, s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_predict_batch(int strict, const PredictBatch& b, long nxyz, int n_items, cudaStream_t s) {
  if (n_items <= 0) return 0;
  dim3 grid((unsigned)((nxyz + 255) / 256), (unsigned)n_items);
  if (strict)
    k_predict_batch<float, true><<<grid, 256, 0, s>>>(b);
  else
    k_predict_batch<float, false><<<grid, 256, 0, s>>>(b);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

bool pencils_batch_maps(int N, int mode, int strict, int qb, PencilArgs* a) {
  const int TX = pencil_tx(N, 1);
  bool ok = encode_stage_map(&a->tm_x, a->xr ? a->xr : (const void*)a->x, !a->xr, N, a->n_qp, TX, qb) &&
            encode_stage_map(&a->tm_t, a->txy, false, N, a->n_qp, TX, qb);
  if (ok && mode == M_CORRECT) {
    ok = encode_stage_map(&a->tm_q, a->q, true, N, a->n_qp, TX, qb) &&
         (strict || encode_stage_map(&a->tm_r, a->r, false, N, a->n_qp, TX, qb));
  }
  return ok;
}

template <typename R, int N>
static int pencils_n(int mode, const PencilArgs& a, cudaStream_t s, int qb) {
  switch (mode) {
    case M_RHS: return pencils_nm<R, N, M_RHS>(a, s, qb);
    case M_TAYLOR_FIRST: return pencils_nm<R, N, M_TAYLOR_FIRST>(a, s, qb);
    case M_TAYLOR: return pencils_nm<R, N, M_TAYLOR>(a, s, qb);
    case M_CORRECT: return pencils_nm<R, N, M_CORRECT>(a, s, qb);
    case M_DERIV_PREDICT: return pencils_nm<R, N, M_DERIV_PREDICT>(a, s, qb);
    case M_ENERGY: return pencils_nm<R, N, M_ENERGY>(a, s, qb);
    case M_ETA: return pencils_nm<R, N, M_ETA>(a, s, qb);
    default: return 1;
  }
}

template <typename R, int N>
static bool qb_valid_n(int qb) {
  if (qb == 1) return pencil_oz<R, N>();
  if (qb == 2) return qb_fits<R, N, 2>();
  if (qb == 4) return qb_fits<R, N, 4>();
  return false;
}

int launch_planes(int N, int mixed, const PlanesArgs& a, cudaStream_t s, int pb) {
  switch (N) {
#define CASE(n) \
  case n: return mixed ? planes_n<float, n>(a, s, pb) : planes_n<double, n>(a, s, pb);
    LISE_FOR_N(CASE)
#undef CASE
    default: return 1;
  }
}

int launch_pencils(int N, int mixed, int mode, const PencilArgs& a, cudaStream_t s, int qb) {
  switch (N) {
#define CASE(n) \
  case n: return mixed ? pencils_n<float, n>(mode, a, s, qb) : pencils_n<double, n>(mode, a, s, qb);
    LISE_FOR_N(CASE)
#undef CASE
    default: return 1;
  }
}

bool planes_pb_valid(int N, int mixed, int pb) {
  switch (N) {
#define CASE(n) \
  case n: return mixed ? planes_pb_valid_n<float, n>(pb) : planes_pb_valid_n<double, n>(pb);
    LISE_FOR_N(CASE)
#undef CASE
    default: return false;
  }
}

int planes_pb(int N, int mixed) {
  const int t = planes_pb_get(N, mixed);
  if (t) return t;
  switch (N) {
#define CASE(n) \
  case n: return PlanesPB<n>::v;
    LISE_FOR_N(CASE)
#undef CASE
    default: return 0;
  }
}

bool pencil_qb_valid(int N, int mixed, int qb) {
  switch (N) {
#define CASE(n) \
  case n: return mixed ? qb_valid_n<float, n>(qb) : qb_valid_n<double, n>(qb);
    LISE_FOR_N(CASE)
#undef CASE
    default: return false;
  }
}

int launch_reduce(const ReduceArgs& a, cudaStream_t s) {
  const int nt = 256;
  const long blocks = (a.nxyz + nt - 1) / nt;
  k_reduce<<<(unsigned)blocks, nt, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_predict(const PointwiseArgs& a, cudaStream_t s) {
  const int nt = 256;
  dim3 grid((unsigned)((a.nxyz + nt - 1) / nt), (a.n_qp + a.qg - 1) / a.qg);
  if (a.mixed && a.strict)
    k_predict<float, true><<<grid, nt, 0, s>>>(a);
  else if (a.mixed)
    k_predict<float><<<grid, nt, 0, s>>>(a);
  else
    k_predict<double><<<grid, nt, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_norms(const double2* y, int n_qp, long nxyz, double a3, int nb, double* part, double* scale,
                 cudaStream_t s) {
  k_norm_part<<<dim3((unsigned)nb, (unsigned)n_qp), 256, 0, s>>>(y, nxyz, nb, part);
  if (cudaGetLastError() != cudaSuccess) return 3;
  k_norm_scale<<<(unsigned)((n_qp + 127) / 128), 128, 0, s>>>(part, n_qp, nb, a3, scale);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_scale_density(double2* y, const double* scale, const PointwiseArgs& a, cudaStream_t s) {
  const int nt = 256;
  dim3 grid((unsigned)((a.nxyz + nt - 1) / nt), (a.n_qp + a.qg - 1) / a.qg);
  k_scale_density<<<grid, nt, 0, s>>>(y, scale, a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_currents(const double2* psi, const double* d1, int N, int n_qp, int qg, double* jx, double* jy,
                    double* jz, cudaStream_t s) {
  const int n_groups = (n_qp + qg - 1) / qg;
  dim3 grid((unsigned)(N * N), (unsigned)n_groups);
  const size_t smem = (size_t)N * (sizeof(double2) + sizeof(double));
  k_currents<<<grid, N, smem, s>>>(psi, d1, N, n_qp, qg, jx, jy, jz);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_sum_groups3(const double* jx, const double* jy, const double* jz, int n_groups, long nxyz, double* out,
                       cudaStream_t s) {
  const int nt = 256;
  k_sum_groups3<<<(unsigned)((nxyz + nt - 1) / nt), nt, 0, s>>>(jx, jy, jz, n_groups, nxyz, out);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

void first_derivative_table(int N, double a, double* d1) {
  const long double PI = 3.141592653589793238462643383279502884L;
  for (int m = 0; m < N; ++m) {
    long double acc = 0;
    for (int j = 0; j < N; ++j) {
      if (N % 2 == 0 && j == N / 2) continue;  // the Nyquist coefficient of an odd derivative
      const long double kj = 2.0L * PI * (long double)(j < N / 2 ? j : j - N) / ((long double)N * a);
      acc += -kj * sinl(kj * (long double)m * a);  // Re(i k e^{i k m a})
    }
    d1[m] = (double)(acc / N);
  }
}

int launch_kick(const double2* src, double2* dst, const double* chi, int n_qp, long nxyz, cudaStream_t s) {
  const long count = (long)n_qp * 2 * nxyz;
  const int nt = 256;
  const long blocks = std::min<long>((count + nt - 1) / nt, 148L * 16);
  if (blocks <= 0) return 0;
  k_kick<<<(unsigned)blocks, nt, 0, s>>>(src, dst, chi, count, nxyz);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_density(const PointwiseArgs& a, cudaStream_t s) {
  const int nt = 256;
  dim3 grid((unsigned)((a.nxyz + nt - 1) / nt), (a.n_qp + a.qg - 1) / a.qg);
  k_density<<<grid, nt, 0, s>>>(a);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

bool ozaki_path(int N, int mixed) { return !mixed && N % 16 == 0 && supported_n(N); }

size_t ozaki_table_words(int N) {
  // mma.sync fragments, then (N = 32, 48: the tcgen05 planes kernels) the core-matrix table
  return (size_t)oz::S * (N / 8) * (N / 16) * 32 * 2 + ((N == 32 || N == 48) ? (size_t)oz::S * N * N / 2 : 0);
}

// D2[n][k] = (1/N) sum_j (alpha/2) k_j^2 cos(k_j (n - k) a), k_j = 2 pi (j or j - N) / (N a),
// as balanced base-256 digits of I_D = round(D2 2^-sD) (|I_D| <= 2^55), laid out as the
// B fragments of mma.m16n8k16 (B[k][n] = D2[n][k]) for each digit, 8-wide output tile,
// k-step and lane: {B[2t][g], B[2t+1][g]}, {B[2t+8][g], B[2t+9][g]}, g = lane / 4, t = lane % 4.
int ozaki_table(int N, double a, double alpha, uint32_t* out) {
  const long double PI = 3.141592653589793238462643383279502884L;
  if (N > 64) return 0;
  long double d[64];  // fixed storage: no heap use (the no-allocation path calls this)
  long double dmax = 0;
  for (int m = 0; m < N; ++m) {
    long double acc = 0;
    for (int j = 0; j < N; ++j) {
      const long double kj = 2.0L * PI * (long double)(j < N / 2 ? j : j - N) / ((long double)N * a);
      acc += 0.5L * alpha * kj * kj * cosl(kj * (long double)m * a);
    }
    d[m] = acc / N;
    dmax = std::max(dmax, fabsl(d[m]));
  }
  int eD = 0;
  while (ldexpl(1.0L, eD) < dmax) ++eD;
  while (eD > -1000 && ldexpl(1.0L, eD - 1) >= dmax) --eD;
  const int sD = eD - 55;
  // digits of every circulant entry
  int dig[oz::S * 64];
  for (int m = 0; m < N; ++m) {
    long long I = llroundl(ldexpl(d[m], -sD));
    int carry = 0;
    for (int k = oz::S - 1; k >= 1; --k) {
      const int byte = (int)((unsigned long long)I >> (8 * (oz::S - 1 - k)) & 0xFFu) + carry;
      carry = (byte + 128) >> 8;
      dig[(size_t)k * N + m] = byte - (carry << 8);
    }
    dig[m] = (int)(I >> 48) + carry;
  }
  auto bf16 = [](int v) -> uint32_t {  // small integer -> bf16 bits (exact)
    const float f = (float)v;
    uint32_t u;
    std::memcpy(&u, &f, 4);
    return u >> 16;
  };
  auto D = [&](int l, int n, int k) { return dig[(size_t)l * N + ((n - k) % N + N) % N]; };
  const int KS = N / 16, NTL = N / 8;
  for (int l = 0; l < oz::S; ++l)
    for (int nt = 0; nt < NTL; ++nt)
      for (int ks = 0; ks < KS; ++ks)
        for (int lane = 0; lane < 32; ++lane) {
          const int g = lane / 4, t = lane % 4, n = nt * 8 + g, k0 = ks * 16 + 2 * t;
          uint32_t* o = out + ((((size_t)l * NTL + nt) * KS + ks) * 32 + lane) * 2;
          o[0] = bf16(D(l, n, k0)) | (bf16(D(l, n, k0 + 1)) << 16);
          o[1] = bf16(D(l, n, k0 + 8)) | (bf16(D(l, n, k0 + 9)) << 16);
        }
  if (N == 32) {
    // [digit][n][k] in the K-major core-matrix layout of the tcgen05 operands (bf16 pairs)
    uint32_t* t = out + (size_t)oz::S * NTL * KS * 32 * 2;
    for (int l = 0; l < oz::S; ++l)
      for (int n = 0; n < N; ++n)
        for (int k = 0; k < N; k += 2) {
          const size_t byte = (size_t)l * N * N * 2 + (size_t)(n / 8) * (N / 8) * 128 + (k / 8) * 128 + (n % 8) * 16 + (k % 8) * 2;
          t[byte / 4] = bf16(D(l, n, k)) | (bf16(D(l, n, k + 1)) << 16);
        }
  }
  if (N == 48) {
    // output-column chunks [0, 32) and [32, 48): [chunk o][digit][n' < width][k] (row l width + n'
    // of chunk o is digit l of D2 row start + n'), K-major core matrices, for the chunked tcgen05
    // planes kernel
    uint32_t* t = out + (size_t)oz::S * NTL * KS * 32 * 2;
    const size_t sbo = (size_t)(N / 8) * 128;
    const int width[2] = {32, 16}, start[2] = {0, 32};
    size_t base = 0;
    for (int o = 0; o < 2; ++o) {
      for (int l = 0; l < oz::S; ++l)
        for (int n1 = 0; n1 < width[o]; ++n1)
          for (int k = 0; k < N; k += 2) {
            const int row = l * width[o] + n1;
            const size_t byte = base + (size_t)(row / 8) * sbo + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2;
            t[byte / 4] = bf16(D(l, start[o] + n1, k)) | (bf16(D(l, start[o] + n1, k + 1)) << 16);
          }
      base += (size_t)oz::S * width[o] * N * 2;
    }
  }
  return sD;
}

double pairing_lattice_c(double a, double alpha) {
  const double PI = 3.14159265358979323846;
  const double K = 2.442749607806335;  // Eq. geff_3D
  return (1.0 / alpha) / (4.0 * PI * PI) * (PI / a) * K;
}

int launch_energy_sites(const double* part_ekin, int n_groups, const double* n, const double2* nu,
                        const double* v_static, double drive, const Pairing& pair, int N, double a,
                        double* e_site, cudaStream_t s) {
  const int nt = 256;
  const long nxyz = (long)N * N * N;
  k_energy_sites<<<(unsigned)((nxyz + nt - 1) / nt), nt, 0, s>>>(part_ekin, n_groups, n, nu, v_static, drive, pair,
                                                                  N, a, e_site);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int launch_eta_reduce(const double* eta_part, int n_qp, int n_blocks, double a3, double* eta, cudaStream_t s) {
  k_eta_reduce<<<(n_qp + 127) / 128, 128, 0, s>>>(eta_part, n_qp, n_blocks, a3, eta);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

int pencil_blocks_x(int N, int mixed) { return (N / pencil_tx(N, mixed)) * N; }

void choose_groups(int N, int n_qp, int mixed, int* qg, int* n_groups) {
  const int tiles = pencil_blocks_x(N, mixed);
  int q = 64;
  while (q > 4 && (long)tiles * ((n_qp + q - 1) / q) < 2048) q /= 2;
  if (q > n_qp) q = n_qp;
  *qg = q;
  *n_groups = (n_qp + q - 1) / q;
}

template <typename R>
static void fft_tables_r(int N, double a, double alpha, R* tw, R* hxy, R* hz) {
  const long double PI = 3.141592653589793238462643383279502884L;
  // twiddles tw[j2 N1 + k1] = exp(-2 pi i (j2 k1 mod N) / N); the four-step plan reads
  // entries with j2 < N2, k1 < N1 only
  int N1 = 0;
  switch (N) {
    case 8: N1 = 2; break;
    case 12: case 16: case 20: case 24: case 32: N1 = 4; break;
    default: N1 = 8; break;
  }
  const int N2 = N / N1;
  for (int j2 = 0; j2 < N2; ++j2)
    for (int k1 = 0; k1 < N1; ++k1) {
      const long e = ((long)j2 * k1) % N;
      const long double ang = -2.0L * PI * (long double)e / (long double)N;
      tw[2 * (j2 * N1 + k1)] = (R)cosl(ang);
      tw[2 * (j2 * N1 + k1) + 1] = (R)sinl(ang);
    }
  const long double L = (long double)N * a;
  for (int k = 0; k < N; ++k) {
    // Sec. "Discretization": k = 2 pi n / L over n = -N/2 .. N/2-1 (index n mod N)
    const long double kk = 2.0L * PI * (long double)(k < N / 2 ? k : k - N) / L;
    const long double f = 0.5L * alpha * kk * kk;
    hxy[k] = (R)(f / ((long double)N * N));
    hz[k] = (R)(f / (long double)N);
  }
}

void fill_fft_tables(int N, double a, double alpha, int mixed, void* tw, void* hxy, void* hz) {
  if (mixed)
    fft_tables_r<float>(N, a, alpha, (float*)tw, (float*)hxy, (float*)hz);
  else
    fft_tables_r<double>(N, a, alpha, (double*)tw, (double*)hxy, (double*)hz);
}

int launch_finite_check(const double2* x, long count, int* err, cudaStream_t s) {
  k_finite<<<148 * 4, 256, 0, s>>>(x, count, err);
  return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // namespace lise
