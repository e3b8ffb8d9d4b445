// pai_row_kernels.cuh -- sm_103a row kernels of the NUFFT Fourier reconstruction.
//
// One "row" is one lateral frequency K_lat of the detector data after the
// lateral FFT (Eq. fft-1a).  For every row the forward kernel performs the
// whole one-dimensional nonuniform FFT of Algorithm 1 plus the weight of
// Eq. (fft-0) without leaving the SM:
//
//   1. prescale (Algorithm 1, division by the window) and zero padding to the
//      oversampled length M = c nt, written straight into shared memory;
//   2. the length-M FFT of Eq. (nufft-c), in shared memory (Stockham
//      autosort, radix 16/8/4/2, each thread holding 16 values in registers
//      per pass; at oversampling 2 the first pass skips the zero padding, as
//      two length-8 DFTs or, for M = 32 16^k, as a radix-32 pass shared by
//      two threads);
//   3. the truncated window gather of Eq. (nufft-a) at the nodes
//      omega = c_s sign(Kz) |K| (Eq. dft-2d), multiplied by the weight of
//      Eq. (fft-0), written to the half image spectrum.
//
// The oversampled spectrum of a row therefore never reaches HBM: a row costs
// one read of its nt complex samples and one write of its nz/2+1 (or twice
// that) spectrum values.  The adjoint kernel runs the exact transpose of the
// same steps in reverse order (spread in gather form, inverse FFT, prescale).
//
// Conventions fixed by the design (each traced to the paper):
//  * the constant of Fourmont's identity is 1/(2 pi c) (it is the Fourier
//    coefficient of a 2 pi c periodic function); it lives in the prescale;
//  * the phase of the Proposition (Eq. nufft-a) is e^{-i pi (omega - j/c)}:
//    the e^{+i pi j/c} part is applied by storing sample n at position
//    n - nt/2 (mod M) before the FFT, the e^{-i pi omega} part once per node;
//  * taps are wrapped modulo M (the oversampled spectrum is M-periodic by
//    Eq. nufft-c), so nodes beyond the Nyquist band are handled exactly;
//  * node positions are computed in float-float arithmetic (about 44
//    significant bits) because an FP32 node alone would cost 1e-5 relative
//    error at |omega| ~ 3000.
#include <cuda_runtime.h>
#include <stdint.h>

#pragma once
#include "pai_internal.h"

namespace pai {

#define PADI(i) ((i) + ((i) >> 5))

// Complex arithmetic on the packed two-lane FP32 instructions of sm_100+
// (add/sub/mul/fma .rn.f32x2): one instruction per complex add, two per
// complex product.  Each lane rounds exactly like its scalar counterpart.
__device__ __forceinline__ unsigned long long pack2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 unpack2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
__device__ __forceinline__ float2 csub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)));
  return unpack2(r);
}
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pack2(a)), "l"(pack2(b)), "l"(pack2(c)));
  return unpack2(r);
}
// (a.x + i a.y)(b.x + i b.y) = a.x (b.x, b.y) + a.y (-b.y, b.x)
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return fma2(make_float2(a.x, a.x), b, mul2(make_float2(a.y, a.y), make_float2(-b.y, b.x)));
}

// cos and sin of 2 pi q / 16, q = 0..7
__host__ __device__ constexpr float cos16(int q) {
  return q == 0 ? 1.0f : q == 1 ? 0.92387953251128674f : q == 2 ? 0.70710678118654752f
       : q == 3 ? 0.38268343236508977f : q == 4 ? 0.0f : q == 5 ? -0.38268343236508977f
       : q == 6 ? -0.70710678118654752f : -0.92387953251128674f;
}
__host__ __device__ constexpr float sin16(int q) {
  return q == 0 ? 0.0f : q == 1 ? 0.38268343236508977f : q == 2 ? 0.70710678118654752f
       : q == 3 ? 0.92387953251128674f : q == 4 ? 1.0f : q == 5 ? 0.92387953251128674f
       : q == 6 ? 0.70710678118654752f : 0.38268343236508977f;
}

// cos and sin of 2 pi q / 32, q = 0..8
__host__ __device__ constexpr float cos32(int q) {
  return q == 0 ? 1.0f : q == 1 ? 0.98078528040323044913f : q == 2 ? 0.92387953251128675613f
       : q == 3 ? 0.83146961230254523708f : q == 4 ? 0.70710678118654752440f : q == 5 ? 0.55557023301960222474f
       : q == 6 ? 0.38268343236508977173f : q == 7 ? 0.19509032201612826785f : 0.0f;
}
__host__ __device__ constexpr float sin32(int q) { return cos32(8 - q); }

// x * e^{-+ 2 pi i q / 32}, q = 0..8  (CONJ: plus sign)
template <int Q, bool CONJ>
__device__ __forceinline__ float2 tw32(float2 x) {
  if (Q == 0) return x;
  if (Q == 8) return CONJ ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
  constexpr float c = cos32(Q);
  constexpr float s = CONJ ? sin32(Q) : -sin32(Q);
  return fma2(make_float2(x.x, x.x), make_float2(c, s), mul2(make_float2(x.y, x.y), make_float2(-s, c)));
}

// x * e^{-+ 2 pi i q / 16}  (forward: minus sign; INV: plus sign)
template <int Q, bool INV>
__device__ __forceinline__ float2 twq(float2 x) {
  if (Q == 0) return x;
  if (Q == 4) return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
  constexpr float c = cos16(Q);
  constexpr float s = INV ? sin16(Q) : -sin16(Q);
  return fma2(make_float2(x.x, x.x), make_float2(c, s), mul2(make_float2(x.y, x.y), make_float2(-s, c)));
}

template <int R>
__host__ __device__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1, k = R >> 1; b < R; b <<= 1, k >>= 1)
    if (i & b) r |= k;
  return r;
}

// Butterfly stage of an in-register radix-2 DIT FFT of size R (data in
// bit-reversed order).  Stage span m, half h = m/2, twiddle q = k * 16/m.
template <int R, int M2, int K, bool INV>
struct Stage {
  __device__ __forceinline__ static void run(float2 (&a)[R]) {
    constexpr int h = M2 / 2;
#pragma unroll
    for (int g = 0; g < R; g += M2) {
      float2 u = a[g + K];
      float2 t = twq<K * (16 / M2), INV>(a[g + K + h]);
      a[g + K] = cadd(u, t);
      a[g + K + h] = csub(u, t);
    }
    Stage<R, M2, K + 1, INV>::run(a);
  }
};
template <int R, int M2, bool INV>
struct Stage<R, M2, M2 / 2, INV> {
  __device__ __forceinline__ static void run(float2 (&)[R]) {}
};

template <int R, int M2, bool INV>
struct Stages {
  __device__ __forceinline__ static void run(float2 (&a)[R]) {
    Stage<R, M2, 0, INV>::run(a);
    Stages<R, M2 * 2, INV>::run(a);
  }
};
template <int R, bool INV>
struct Stages<R, R * 2, INV> {
  __device__ __forceinline__ static void run(float2 (&)[R]) {}
};

// v <- DFT_R(v): v[k] = sum_r v[r] e^{-+ 2 pi i r k / R}
template <int R, bool INV>
__device__ __forceinline__ void dft_reg(float2 (&v)[R]) {
  float2 a[R];
#pragma unroll
  for (int i = 0; i < R; ++i) a[bitrev<R>(i)] = v[i];
  Stages<R, 2, INV>::run(a);
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = a[i];
}

// Layouts of a row slot in shared memory.  Passes between the first and the
// last keep one padding element every 32 (PADI) so strided butterfly accesses
// do not collide in the banks.  The last pass of the forward transform writes
// the spectrum unpadded and repeats its first 2*kMaxH values after index M
// ("ghost cells"), so a node's 2H consecutive taps are plain consecutive
// addresses even when the window wraps around the period M.
enum : int { kLayoutPadded = 0, kLayoutFlat = 1, kLayoutFlatGhost = 2 };

// One in-place Stockham pass of radix R.  Butterfly j (0 <= j < M/R) reads
// X[j + r M/R], twiddles by e^{-+2 pi i r (j mod Ns) / (Ns R)}, and writes its
// R outputs to X[(j - j mod Ns) R + (j mod Ns) + r Ns].  All reads of the
// pass complete (barrier) before any write.  OUT selects the write layout.
// Twiddle powers w^1 .. w^(R-1) from the table entries w^1, w^2, w^4, w^8
// (loaded before the pass barrier); the others are products of at most
// three of them, so each power carries at most three extra roundings.
template <int R>
struct TwBase {
  float2 b[R >= 16 ? 4 : R >= 8 ? 3 : R >= 4 ? 2 : 1];
};

// The twiddle table is two-level (twiddle_table): w^k = hi[k >> 6] lo[k & 63]
// with lo = tw[0..63] and hi = tw[64..], w = e^{-2 pi i / TW}.  Both parts
// together hold 64 + TW/64 values (2.5 KB at TW = 16384), so they stay in L1
// while a full-length table (64 KB at TW = 8192) would miss there; the
// product costs one complex multiply and about one extra rounding.
__device__ __forceinline__ float2 tw_at(const float2* __restrict__ tw, int k) {
  return cmul(__ldg(&tw[kTwLo + (k >> kTwLoShift)]), __ldg(&tw[k & (kTwLo - 1)]));
}

template <int R>
__device__ __forceinline__ void tw_load(TwBase<R>& t, const float2* __restrict__ tw, int step) {
  t.b[0] = tw_at(tw, step);
  if (R >= 4) t.b[1] = tw_at(tw, 2 * step);
  if (R >= 8) t.b[2] = tw_at(tw, 4 * step);
  if (R >= 16) t.b[3] = tw_at(tw, 8 * step);
}

// x * e^{-2 pi i q / 16}, q = 0..15 (a constant once the caller's loop is unrolled)
__device__ __forceinline__ float2 rot16(float2 x, int q) {
  const float c = (q & 8) ? -cos16(q & 7) : cos16(q & 7);
  const float s = (q & 8) ? sin16(q & 7) : -sin16(q & 7);
  return fma2(make_float2(x.x, x.x), make_float2(c, s), mul2(make_float2(x.y, x.y), make_float2(-s, c)));
}

// Base twiddles of butterfly j + i M/16 from those of butterfly j, for the last
// pass of a transform (Ns R = M, so the twiddle index is the butterfly index):
// w^{2^e (j + i M/16)} = w^{2^e j} e^{-2 pi i (2^e i mod 16) / 16}.
template <int R>
__device__ __forceinline__ void tw_shift(TwBase<R>& t, const TwBase<R>& t0, int i) {
  t.b[0] = rot16(t0.b[0], i & 15);
  if (R >= 4) t.b[1] = rot16(t0.b[1], (2 * i) & 15);
  if (R >= 8) t.b[2] = rot16(t0.b[2], (4 * i) & 15);
  if (R >= 16) t.b[3] = rot16(t0.b[3], (8 * i) & 15);
}

template <bool INV>
__device__ __forceinline__ float2 twc(float2 w) {
  return INV ? make_float2(w.x, -w.y) : w;
}

// v[r] *= w^r for r = 1..R-1, each power formed right before its use so only
// the base entries stay live.
template <int R, bool INV>
__device__ __forceinline__ void tw_apply(float2 (&v)[R], const TwBase<R>& t) {
  const float2 w1 = t.b[0];
  v[1] = cmul(v[1], twc<INV>(w1));
  if (R >= 4) {
    const float2 w2 = t.b[1];
    const float2 w3 = cmul(w1, w2);
    v[2] = cmul(v[2], twc<INV>(w2));
    v[3] = cmul(v[3], twc<INV>(w3));
    if (R >= 8) {
      const float2 w4 = t.b[2];
      const float2 w5 = cmul(w1, w4), w6 = cmul(w2, w4), w7 = cmul(w3, w4);
      v[4] = cmul(v[4], twc<INV>(w4));
      v[5] = cmul(v[5], twc<INV>(w5));
      v[6] = cmul(v[6], twc<INV>(w6));
      v[7] = cmul(v[7], twc<INV>(w7));
      if (R >= 16) {
        const float2 w8 = t.b[3];
        v[8] = cmul(v[8], twc<INV>(w8));
        v[9] = cmul(v[9], twc<INV>(cmul(w1, w8)));
        v[10] = cmul(v[10], twc<INV>(cmul(w2, w8)));
        v[11] = cmul(v[11], twc<INV>(cmul(w3, w8)));
        v[12] = cmul(v[12], twc<INV>(cmul(w4, w8)));
        v[13] = cmul(v[13], twc<INV>(cmul(w5, w8)));
        v[14] = cmul(v[14], twc<INV>(cmul(w6, w8)));
        v[15] = cmul(v[15], twc<INV>(cmul(w7, w8)));
      }
    }
  }
}

// Padded addresses without per-element shifts: for a multiple S of 32,
// PADI(a + r S) = PADI(a) + r (S + S/32); and for a with a mod 32 < 16,
// PADI(a + 16 r) = PADI(a) + 16 r + r/2 (r < 16).  Both hold for every pass
// after the first radix-16 one (Ns = 16 or a multiple of 256), and for the
// first pass (Ns = 1) PADI(16 j + r) = PADI(16 j) + r.
// CHAIN_R: the smallest radix whose last pass derives its twiddles by
// rotation (tw_shift); below it they come from the table.
template <int R, bool INV, int OUT, int CHAIN_R = 2>
__device__ __forceinline__ void fft_pass(float2* X, int M, int Ns, int lane, int tpr, const float2* __restrict__ tw,
                                         int twstride, bool active = true) {
  constexpr int NB = kElemsPerThread / R;
  float2 v[NB][R];
  TwBase<R> t[NB];
  const int MR = M / R;
  const int tws = (M / (Ns * R)) * twstride;
  // A last pass of radix < 16 (several butterflies per thread, at j = lane +
  // i M/16): their twiddles follow from the first butterfly's by constant
  // rotations (tw_shift) instead of table loads.
  const bool chain = R >= CHAIN_R && NB > 1 && Ns > 1 && Ns * R == M && tpr * kElemsPerThread == M;
  // twiddles do not depend on the data: for radix 16 (one butterfly per
  // thread) their loads are issued before the barrier; smaller radices carry
  // several butterflies per thread and load after it to stay within registers
  if (active) {
    if (Ns > 1 && NB == 1) tw_load<R>(t[0], tw, (lane & (Ns - 1)) * tws);
    if ((MR & 31) == 0) {
      const int rs = MR + (MR >> 5);
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const float2* src = X + PADI(lane + i * tpr);
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = src[r * rs];
      }
    } else {
#pragma unroll
      for (int i = 0; i < NB; ++i) {
        const int j = lane + i * tpr;
#pragma unroll
        for (int r = 0; r < R; ++r) v[i][r] = X[PADI(j + r * MR)];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (!active) break;
    const int j = lane + i * tpr;
    const int k = j & (Ns - 1);
    if (Ns > 1) {
      if (NB != 1) {
        if (!chain || i == 0) tw_load<R>(t[i], tw, k * tws);
        else tw_shift<R>(t[i], t[0], i);
      }
      tw_apply<R, INV>(v[i], t[i]);
    }
    dft_reg<R, INV>(v[i]);
    const int base = (j - k) * R + k;
    if (OUT == kLayoutPadded) {
      float2* dst = X + PADI(base);
      if (Ns == 16) {
#pragma unroll
        for (int r = 0; r < R; ++r) dst[16 * r + (r >> 1)] = v[i][r];
      } else if ((Ns & 31) == 0) {
        const int ws = Ns + (Ns >> 5);
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r * ws] = v[i][r];
      } else if (Ns == 1 && R == 16) {
#pragma unroll
        for (int r = 0; r < R; ++r) dst[r] = v[i][r];
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) X[PADI(base + r * Ns)] = v[i][r];
      }
    } else {
      float2* dst = X + base;
#pragma unroll
      for (int r = 0; r < R; ++r) dst[r * Ns] = v[i][r];
      if (OUT == kLayoutFlatGhost && base < 2 * kMaxH) {
#pragma unroll
        for (int r = 0; r < R; ++r)
          if (base + r * Ns < 2 * kMaxH) X[M + base + r * Ns] = v[i][r];
      }
    }
  }
  __syncthreads();
}

// Sample n of a row's lateral spectrum: src[n], or (paired layout, see
// RowProblem::paired) separated from the transforms of the sample pairs,
// z1 = Z[k][m], z2 = Z[nx - k][m] with m = n/2:
// sample 2m = (z1 + conj z2) / 2, sample 2m+1 = (z1 - conj z2) / (2i).
template <bool PAIRED>
__device__ __forceinline__ float2 row_sample(const float2* __restrict__ src, const float2* __restrict__ src2, int n) {
  if (!PAIRED) return __ldg(&src[n]);
  const float2 z1 = __ldg(&src[n >> 1]), z2 = __ldg(&src2[n >> 1]);
  return (n & 1) ? make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x))
                 : make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
}

// First forward pass (radix 16, Ns = 1) fed straight from global memory:
// position m = j + r M/16 of the oversampled input holds sample
// n = m + nt/2 (mod M) times the prescale when n < nt, else zero (Algorithm 1
// prescale and zero padding, centred so that the e^{+i pi j/c} part of the
// Proposition's phase is absorbed).  Writes padded.
template <bool PAIRED = false>
__device__ __forceinline__ void fft_first_pass_from_global(float2* X, int M, int nt, int lane, int tpr,
                                                           const float2* __restrict__ src,
                                                           const float* __restrict__ prescale,
                                                           const float2* __restrict__ src2 = nullptr) {
  constexpr int R = 16;
  float2 v[R];
  const int MR = M / R, mask = M - 1, h = nt >> 1;
  if (M == 2 * nt) {
    // Oversampling 2: only the inputs r = 0..3 and 12..15 hold samples (the
    // others fall in the zero padding), a block b_s, s = -4..3, of 8 values.
    // With w = e^{-2 pi i/16}: X[2m] = sum_s b_s w^{2sm} and
    // X[2m+1] = sum_s (b_s w^s) w^{2sm}, two length-8 DFTs.
    float2 c8[8], d8[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int r = q < 4 ? q : q + 8;
      const int n = (lane + r * MR + h) & mask;
      const float2 g = row_sample<PAIRED>(src, src2, n);
      const float s = __ldg(&prescale[n]);
      c8[q] = make_float2(s * g.x, s * g.y);
    }
    d8[0] = c8[0];
    d8[1] = twq<1, false>(c8[1]);
    d8[2] = twq<2, false>(c8[2]);
    d8[3] = twq<3, false>(c8[3]);
    d8[4] = twq<4, true>(c8[4]);  // w^-4 = i
    d8[5] = twq<3, true>(c8[5]);
    d8[6] = twq<2, true>(c8[6]);
    d8[7] = twq<1, true>(c8[7]);
    dft_reg<8, false>(c8);
    dft_reg<8, false>(d8);
    float2* dst = X + PADI(lane * R);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      dst[2 * m] = c8[m];
      dst[2 * m + 1] = d8[m];
    }
    __syncthreads();
    return;
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int m = lane + r * MR;
    const int n = (m + h) & mask;
    float2 a = make_float2(0.f, 0.f);
    if (n < nt) {
      const float2 g = row_sample<PAIRED>(src, src2, n);
      const float s = __ldg(&prescale[n]);
      a = make_float2(s * g.x, s * g.y);
    }
    v[r] = a;
  }
  dft_reg<R, false>(v);
  float2* dst = X + PADI(lane * R);
#pragma unroll
  for (int r = 0; r < R; ++r) dst[r] = v[r];
  __syncthreads();
}

// First forward pass of radix 32 at oversampling 2 when M = 32 16^k: the
// transform then takes radix-16 passes only (no radix-2 pass at its end).
// Butterfly j (0 <= j < M/32) has inputs x_r at positions j + r M/32, which
// hold samples for r = 0..7 and r = 24..31 only (the rest is padding), and
// outputs X[32 j + q].  Two threads share it: h = 0 computes the even outputs
// X[32 j + 2m] = sum_s z_s w16^{sm} with z_s = x_s + x_{s+16}, h = 1 the odd
// ones with z_s = (x_s - x_{s+16}) w32^s, w_N = e^{-2 pi i/N}; of each pair
// x_s, x_{s+16} one is padding (s < 8: x_{s+16}; s >= 8: x_s).  Both threads
// load the butterfly's 16 samples.  Writes padded: PADI(32 j + q) = 33 j + q.
template <bool PAIRED>
__device__ __forceinline__ void fft_first_pass32_from_global(float2* X, int M, int nt, int lane, int tpr,
                                                             const float2* __restrict__ src,
                                                             const float* __restrict__ prescale,
                                                             const float2* __restrict__ src2) {
  const int half = tpr >> 1, q4 = M >> 2, M32 = M >> 5;
  const int h = lane >= half ? 1 : 0;
  const int j = lane - h * half;
  float2 v[16];
#pragma unroll
  for (int s = 0; s < 16; ++s) {
    const int n = s < 8 ? j + s * M32 + q4 : j + (s - 8) * M32;
    const float2 g = row_sample<PAIRED>(src, src2, n);
    const float p = __ldg(&prescale[n]);
    v[s] = make_float2(p * g.x, p * g.y);
  }
  if (h) {
    v[1] = tw32<1, false>(v[1]);
    v[2] = tw32<2, false>(v[2]);
    v[3] = tw32<3, false>(v[3]);
    v[4] = tw32<4, false>(v[4]);
    v[5] = tw32<5, false>(v[5]);
    v[6] = tw32<6, false>(v[6]);
    v[7] = tw32<7, false>(v[7]);
    // s >= 8: -w32^s = conj(w32^{16-s})
    v[8] = tw32<8, true>(v[8]);
    v[9] = tw32<7, true>(v[9]);
    v[10] = tw32<6, true>(v[10]);
    v[11] = tw32<5, true>(v[11]);
    v[12] = tw32<4, true>(v[12]);
    v[13] = tw32<3, true>(v[13]);
    v[14] = tw32<2, true>(v[14]);
    v[15] = tw32<1, true>(v[15]);
  }
  dft_reg<16, false>(v);
  float2* dst = X + 33 * j + h;
#pragma unroll
  for (int m = 0; m < 16; ++m) dst[2 * m] = v[m];
  __syncthreads();
}

// Whether the forward transform of a row starts with the radix-32 pass.
__device__ __forceinline__ bool first_pass32(int M, int mshift, int nt) {
  return M == 2 * nt && mshift >= 9 && ((mshift - 5) & 3) == 0;
}

// Remaining passes after a first pass of radix 2^ns_shift (16 or 32: Ns on
// entry); the last pass writes layout OUT.
template <bool INV, int OUT, int CHAIN_R = 2>
__device__ __forceinline__ void fft_rest(float2* X, int M, int mshift, int lane, int tpr, const float2* tw,
                                         int twstride, bool active = true, int ns_shift = 4) {
  int Ns = 1 << ns_shift;
  int rem = mshift - ns_shift;
  while (rem >= 4) {
    if (rem == 4) {
      fft_pass<16, INV, OUT>(X, M, Ns, lane, tpr, tw, twstride, active);
      return;
    }
    fft_pass<16, INV, kLayoutPadded>(X, M, Ns, lane, tpr, tw, twstride, active);
    Ns <<= 4;
    rem -= 4;
  }
  if (rem == 3) fft_pass<8, INV, OUT, CHAIN_R>(X, M, Ns, lane, tpr, tw, twstride, active);
  else if (rem == 2) fft_pass<4, INV, OUT, CHAIN_R>(X, M, Ns, lane, tpr, tw, twstride, active);
  else if (rem == 1) fft_pass<2, INV, OUT, CHAIN_R>(X, M, Ns, lane, tpr, tw, twstride, active);
}

// Inverse length-M transform of an adjoint row with the crop fused: the
// passes run remainder radix first and radix 16 last, and the last pass
// (Ns = M/16, butterfly j = lane, outputs at positions m = j + r M/16) writes
// the outputs that hold samples n = (m + nt/2) mod M < nt, times
// s_n = scale * prescale[n], straight to dst[n].  At oversampling 2
// (M = 2 nt) only r = 0..3 (n = m + M/4) and r = 12..15 (n = m - 3M/4) are
// kept, and only those 8 outputs are computed: with w = e^{+2 pi i/16},
// A = inverse DFT8 of the even inputs and B of the odd,
// Y[t] = A[t] + w^t B[t] (t = 0..3) and Y[t+8] = A[t] - w^t B[t] (t = 4..7).
__device__ __forceinline__ void fft_inverse_crop(float2* X, int M, int mshift, int nt, int lane, int tpr,
                                                 const float2* __restrict__ tw, int twstride, float2* dst,
                                                 const float* __restrict__ prescale, float scale, bool valid) {
  int Ns = 1;
  const int r0 = mshift & 3;
  if (r0 == 3) {
    fft_pass<8, true, kLayoutPadded>(X, M, 1, lane, tpr, tw, twstride);
    Ns = 8;
  } else if (r0 == 2) {
    fft_pass<4, true, kLayoutPadded>(X, M, 1, lane, tpr, tw, twstride);
    Ns = 4;
  } else if (r0 == 1) {
    fft_pass<2, true, kLayoutPadded>(X, M, 1, lane, tpr, tw, twstride);
    Ns = 2;
  }
  while (Ns * 16 < M) {
    fft_pass<16, true, kLayoutPadded>(X, M, Ns, lane, tpr, tw, twstride);
    Ns <<= 4;
  }
  if (!valid) return;
  const int j = lane;
  float2 v[16];
  if ((Ns & 31) == 0) {
    const float2* src = X + PADI(j);
    const int rs = Ns + (Ns >> 5);
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = src[r * rs];
  } else {
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = X[PADI(j + r * Ns)];
  }
  if (Ns > 1) {
    TwBase<16> tb;
    tw_load<16>(tb, tw, j * twstride);
    tw_apply<16, true>(v, tb);
  }
  const int q4 = M >> 2;
  if (M == 2 * nt) {
    float2 a[8], b[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      a[q] = v[2 * q];
      b[q] = v[2 * q + 1];
    }
    dft_reg<8, true>(a);
    dft_reg<8, true>(b);
    b[1] = twq<1, true>(b[1]);
    b[2] = twq<2, true>(b[2]);
    b[3] = twq<3, true>(b[3]);
    b[4] = twq<4, true>(b[4]);
    b[5] = twq<5, true>(b[5]);
    b[6] = twq<6, true>(b[6]);
    b[7] = twq<7, true>(b[7]);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const float2 y = q < 4 ? cadd(a[q], b[q]) : csub(a[q], b[q]);
      const int n = q < 4 ? j + q * Ns + q4 : j + (q + 8) * Ns - 3 * q4;
      const float s = scale * __ldg(&prescale[n]);
      dst[n] = make_float2(s * y.x, s * y.y);
    }
    return;
  }
  dft_reg<16, true>(v);
  const int mask = M - 1, h = nt >> 1;
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int n = (j + r * Ns + h) & mask;
    if (n < nt) {
      const float s = scale * __ldg(&prescale[n]);
      dst[n] = make_float2(s * v[r].x, s * v[r].y);
    }
  }
}

// Length-M FFT (M = 2^mshift >= 32) of a padded row slot, in shared memory;
// the last pass writes layout OUT.
// Threads with active == false take part in the barriers only (used when a
// shorter transform runs on a row slot sized for a longer one).
template <bool INV, int OUT>
__device__ __forceinline__ void fft_smem(float2* X, int M, int mshift, int lane, int tpr, const float2* tw,
                                         int twstride, bool active = true) {
  fft_pass<16, INV, kLayoutPadded>(X, M, 1, lane, tpr, tw, twstride, active);
  fft_rest<INV, OUT>(X, M, mshift, lane, tpr, tw, twstride, active);
}

// ---------------------------------------------------------------------------
// Node position x = c omega = B sqrt(S + az) in float-float arithmetic.
// Returns j0 = floor(x), fr = x - j0 in [0,1), and x0 = FP32 value of x.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void node_position(float2 S, float4 zt, float B2hi, float B2lo, int& j0, float& fr,
                                              float& rx) {
  // s = S + az (two-sum of the high parts, low parts added)
  float s_hi = __fadd_rn(S.x, zt.x);
  float bb = __fsub_rn(s_hi, S.x);
  float err = __fadd_rn(__fsub_rn(S.x, __fsub_rn(s_hi, bb)), __fsub_rn(zt.x, bb));
  float s_lo = __fadd_rn(err, __fadd_rn(S.y, zt.y));
  float t = __fadd_rn(s_hi, s_lo);
  s_lo = __fsub_rn(s_lo, __fsub_rn(t, s_hi));
  s_hi = t;
  // y = B^2 s
  float p = __fmul_rn(B2hi, s_hi);
  float e = fmaf(B2hi, s_hi, -p);
  e = fmaf(B2hi, s_lo, e);
  e = fmaf(B2lo, s_hi, e);
  float y_hi = __fadd_rn(p, e);
  float y_lo = __fsub_rn(e, __fsub_rn(y_hi, p));
  // x = sqrt(y): an FP32 root from the reciprocal square root (a few ulp)
  // plus one Newton correction from the exact residual, which leaves about
  // 44 bits; rx = 1/x to FP32 accuracy is the caller's (x = 0 only for the
  // zero-frequency node, where rx = 0)
  rx = y_hi > 0.0f ? rsqrtf(y_hi) : 0.0f;
  const float x0 = y_hi * rx;
  float q = __fmul_rn(x0, x0);
  float qe = fmaf(x0, x0, -q);
  float r = __fadd_rn(__fsub_rn(__fsub_rn(y_hi, q), qe), y_lo);
  float delta = 0.5f * r * rx;
  float fl = floorf(x0);
  j0 = (int)fl;
  fr = __fadd_rn(__fsub_rn(x0, fl), delta);
  if (fr < 0.0f) {
    fr += 1.0f;
    j0 -= 1;
  } else if (fr >= 1.0f) {
    fr -= 1.0f;
    j0 += 1;
  }
}

// The mirrored node -x = (-j0p - 1) + (1 - frp).  For an integer node fr = 1:
// the tap polynomials cover z = fr - 1/2 in [-1/2, 1/2] with both ends, and
// this is the tap set the forward pair evaluation (node_value_pair) uses.
__device__ __forceinline__ void negate_node(int j0p, float frp, int& j0, float& fr) {
  j0 = -j0p - 1;
  fr = 1.0f - frp;
}

// e^{+i pi nu} for nu = (j0 + fr) nt / M, returned as (cos, sin).
// The integer part is reduced exactly: pi j0 nt / M modulo 2 pi is
// pi m2 / M with m2 = j0 nt mod 2M.  When M = 2 nt that angle is a multiple of
// pi/2 and becomes an exact quarter-turn rotation.
__device__ __forceinline__ float2 node_phase(int j0, float fr, int nt, int M, float nt_over_M) {
  float s2, c2;
  sincospif(fr * nt_over_M, &s2, &c2);
  if (M == 2 * nt) {
    // multiply (c2, s2) by i^(j0 mod 4) with selects, no divergent branch
    const int q = j0 & 3;
    float a = (q & 1) ? -s2 : c2;
    float b = (q & 1) ? c2 : s2;
    if (q & 2) {
      a = -a;
      b = -b;
    }
    return make_float2(a, b);
  }
  const int m2 = (int)(((long long)j0 * (long long)nt) & (2LL * M - 1));
  float s1, c1;
  sincospif((float)m2 / (float)M, &s1, &c1);
  return make_float2(c1 * c2 - s1 * s2, s1 * c2 + c1 * s2);
}

// All 2H tap weights of a node with fraction fr (constant-bank coefficients).
template <int H>
__device__ __forceinline__ void tap_weights(const WindowPoly& W, float fr, float (&w)[2 * H]) {
  const float z = fr - 0.5f, z2 = z * z;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
    for (int e = kHalfCoef - 2; e >= 0; --e) {
      E = fmaf(E, z2, W.ce[p][e]);
      O = fmaf(O, z2, W.co[p][e]);
    }
    w[p] = fmaf(z, O, E);
    w[2 * H - 1 - p] = fmaf(-z, O, E);
  }
}

// P(nu) = e^{-i pi nu} sum_t w_t G[(j0 + t) mod M], t = -H+1..H   (Eq. nufft-a).
// U is the flat spectrum with ghost cells: the 2H taps are U[b .. b+2H-1],
// b = (j0 - H + 1) mod M.  Weights are formed pair by pair (tap it and its
// mirror 2H-1-it) and consumed at once.
template <int H>
__device__ __forceinline__ float2 node_value(const float2* U, const WindowPoly& W, int j0, float fr, int M, int nt,
                                             float nt_over_M) {
  const float2* g = U + ((j0 - H + 1) & (M - 1));
  const float z = fr - 0.5f, z2 = z * z;
  float ax = 0.0f, ay = 0.0f;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
    for (int e = kHalfCoef - 2; e >= 0; --e) {
      E = fmaf(E, z2, W.ce[p][e]);
      O = fmaf(O, z2, W.co[p][e]);
    }
    const float wl = fmaf(z, O, E), wh = fmaf(-z, O, E);
    const float2 gl = g[p], gh = g[2 * H - 1 - p];
    ax = fmaf(wl, gl.x, ax);
    ay = fmaf(wl, gl.y, ay);
    ax = fmaf(wh, gh.x, ax);
    ay = fmaf(wh, gh.y, ay);
  }
  const float2 ph = node_phase(j0, fr, nt, M, nt_over_M);
  return make_float2(fmaf(ax, ph.x, ay * ph.y), fmaf(ay, ph.x, -ax * ph.y));
}

// Interpolation methods of Sec. 4 (no window, prescale 1): the oversampled DFT
// D_j = sum_n e^{-2 pi i j n / M} g_n sits on the grid nu_j = j nt / M, and the
// centred spectrum holds U[j] = e^{+i pi nu_j} D_j, so D_j = e^{-i pi nu_j} U[j mod M].
// LINEAR: (1 - fr) D_j0 + fr D_{j0+1};  NEAREST: D_{j0 + (fr >= 1/2)}.
__device__ __forceinline__ float2 grid_value(const float2* U, int j, int M, int nt, float nt_over_M) {
  const float2 u = U[j & (M - 1)];
  const float2 ph = node_phase(j, 0.0f, nt, M, nt_over_M);
  return make_float2(fmaf(u.x, ph.x, u.y * ph.y), fmaf(u.y, ph.x, -u.x * ph.y));
}

__device__ __forceinline__ float2 node_interp(const float2* U, int method, int j0, float fr, int M, int nt,
                                              float nt_over_M) {
  if (method == PAI_METHOD_NEAREST) return grid_value(U, j0 + (fr >= 0.5f ? 1 : 0), M, nt, nt_over_M);
  const float2 a = grid_value(U, j0, M, nt, nt_over_M);
  const float2 b = grid_value(U, j0 + 1, M, nt, nt_over_M);
  return make_float2(fmaf(fr, b.x - a.x, a.x), fmaf(fr, b.y - a.y, a.y));
}

// The value at a node by the problem's method.  Interpolation plans always run
// with H = 2, so the other instantiations carry no method branch.
template <int H>
__device__ __forceinline__ float2 node_eval(const RowProblem& P, const float2* U, const WindowPoly& W, int j0,
                                            float fr) {
  if constexpr (H == 2) {
    if (P.method >= PAI_METHOD_LINEAR) return node_interp(U, P.method, j0, fr, P.M, P.nt, P.nt_over_M);
  }
  return node_value<H>(U, W, j0, fr, P.M, P.nt, P.nt_over_M);
}

struct RowGeom {
  int d1, d2;     // destination rows (full lateral index) of +nu and -nu nodes
  bool mirror;    // row is not self-conjugate: both destinations are written
  float2 S;       // |K_lat/2pi|^2 as float-float
};

__device__ __forceinline__ RowGeom row_geom(const RowProblem& P, int row) {
  RowGeom g;
  const int half = P.n2 >> 1;
  const int i1 = row / (half + 1);
  const int i2 = row - i1 * (half + 1);
  g.mirror = (i2 > 0) && (i2 < half);
  g.d1 = i1 * P.n2 + i2;
  g.d2 = ((P.n1 - i1) % P.n1) * P.n2 + ((P.n2 - i2) % P.n2);
  g.S = P.rowS[row];
  return g;
}

// Node task i of a row: positive l' (1..nz/2-1), negative l' (mirror rows),
// and one Nyquist task evaluating both nodes at |l'| = nz/2.
__device__ __forceinline__ void node_task(int i, int nzh, int nA, int& lp, bool& neg, bool& nyq) {
  neg = false;
  nyq = false;
  if (i < nzh - 1) {
    lp = i + 1;
  } else if (i == nA - 1) {
    lp = nzh;
    nyq = true;
  } else {
    lp = i - (nzh - 1) + 1;
    neg = true;
  }
}

// Values at the node pair +x and -x (x = c nu = j0 + fr, fr in [0, 1)) from one
// evaluation of the tap polynomials.  The mirrored node is taken as
// -x = (-j0 - 1) + (1 - fr): its offset z' = (1 - fr) - 1/2 = -z, so its tap q
// weighs w_q(-z) = w_{2H-1-q}(z) (phi is even), and its phase
// e^{-i pi (-nu)} is the conjugate of the phase of +x.  Both values come out
// exactly as node_eval would give them for the two nodes, without rounding
// 1 - fr.
template <int H>
__device__ __forceinline__ void node_value_pair(const RowProblem& P, const float2* U, const WindowPoly& W, int j0,
                                                float fr, float2& vp, float2& vn) {
  if constexpr (H == 2) {
    if (P.method >= PAI_METHOD_LINEAR) {
      vp = node_interp(U, P.method, j0, fr, P.M, P.nt, P.nt_over_M);
      vn = node_interp(U, P.method, -j0 - 1, 1.0f - fr, P.M, P.nt, P.nt_over_M);
      return;
    }
  }
  const int mask = P.M - 1;
  const float2* gp = U + ((j0 - H + 1) & mask);
  const float2* gn = U + ((-j0 - H) & mask);
  const float z = fr - 0.5f, z2 = z * z;
  float ax = 0.0f, ay = 0.0f, bx = 0.0f, by = 0.0f;
#pragma unroll
  for (int p = 0; p < H; ++p) {
    float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
    for (int e = kHalfCoef - 2; e >= 0; --e) {
      E = fmaf(E, z2, W.ce[p][e]);
      O = fmaf(O, z2, W.co[p][e]);
    }
    const float wl = fmaf(z, O, E), wh = fmaf(-z, O, E);
    const float2 pl = gp[p], ph = gp[2 * H - 1 - p];
    const float2 nl = gn[p], nh = gn[2 * H - 1 - p];
    ax = fmaf(wl, pl.x, ax);
    ay = fmaf(wl, pl.y, ay);
    ax = fmaf(wh, ph.x, ax);
    ay = fmaf(wh, ph.y, ay);
    bx = fmaf(wh, nl.x, bx);
    by = fmaf(wh, nl.y, by);
    bx = fmaf(wl, nh.x, bx);
    by = fmaf(wl, nh.y, by);
  }
  const float2 ph = node_phase(j0, fr, P.nt, P.M, P.nt_over_M);
  vp = make_float2(fmaf(ax, ph.x, ay * ph.y), fmaf(ay, ph.x, -ax * ph.y));
  vn = make_float2(fmaf(bx, ph.x, -by * ph.y), fmaf(by, ph.x, bx * ph.y));
}

// Half image spectrum of one row (ZF = false layout): for l' = 1 .. nz/2 one
// task evaluates the node pair +-|K|; destination row d1 takes the +nu value,
// the conjugate row d2 (mirror rows only) the conjugate of the -nu value, and
// the Nyquist entry l' = nz/2 the mean of both (reading of the l = -nz/2 row).
// Self-conjugate rows (no mirror) need the -nu value only at the Nyquist entry.
template <int H>
__device__ __forceinline__ void gather_row(const RowProblem& P, const WindowPoly& W, const float2* X, int row,
                                           int lane) {
  const RowGeom rg = row_geom(P, row);
  const int nzh = P.nz >> 1;
  float2* out1 = P.fh + (size_t)rg.d1 * P.lz;
  float2* out2 = P.fh + (size_t)rg.d2 * P.lz;
  if (lane == 0) {
    out1[0] = make_float2(0.f, 0.f);
    if (rg.mirror) out2[0] = make_float2(0.f, 0.f);
  }
  // the depth-table entry of the next task is loaded one iteration ahead
  float4 zt_next = __ldg(&P.zt[min(lane, nzh - 1) + 1]);
  for (int i = lane; i < nzh; i += P.tpr) {
    const int lp = i + 1;
    const float4 zt = zt_next;
    if (i + P.tpr < nzh) zt_next = __ldg(&P.zt[lp + P.tpr]);
    int j0;
    float fr, rx;
    node_position(rg.S, zt, P.B2hi, P.B2lo, j0, fr, rx);
    const float wt = P.wscale * zt.z * rx;
    if (lp == nzh || rg.mirror) {
      float2 v, u;
      node_value_pair<H>(P, X, W, j0, fr, v, u);
      if (lp == nzh) {
        const float2 a = make_float2(0.5f * wt * (v.x + u.x), 0.5f * wt * (v.y + u.y));
        out1[lp] = a;
        if (rg.mirror) out2[lp] = make_float2(a.x, -a.y);
      } else {
        out1[lp] = make_float2(wt * v.x, wt * v.y);
        out2[lp] = make_float2(wt * u.x, -wt * u.y);
      }
    } else {
      const float2 v = node_eval<H>(P, X, W, j0, fr);
      out1[lp] = make_float2(wt * v.x, wt * v.y);
    }
  }
}

// Depth-row layout: the row's own full depth spectrum F[l], l in
// [-nz/2, nz/2), stored at Zs[l mod nz] (Zs = the row's line of the output),
// from the row's nodes at +nu (l > 0) and -nu (l < 0):  F[l] = W P(sign(l)|K|)
// for 0 < |l| < nz/2, F[0] = 0 (l = 0 rule), F[-nz/2] = W (P(+|K|) + P(-|K|))/2
// (Nyquist rule).  One task per |l| evaluates the node pair.  An inverse depth
// FFT of each line followed by the lateral C2R completes Eq. (fft-1).
template <int H>
__device__ __forceinline__ void gather_row_z(const RowProblem& P, const WindowPoly& W, const float2* X, float2* Zs,
                                             int row, int lane) {
  const float2 S = P.rowS[row];
  const int nzh = P.nz >> 1;
  if (lane == 0) Zs[0] = make_float2(0.f, 0.f);
  float4 zt_next = __ldg(&P.zt[min(lane, nzh - 1) + 1]);
  for (int i = lane; i < nzh; i += P.tpr) {
    const int lp = i + 1;
    const float4 zt = zt_next;
    if (i + P.tpr < nzh) zt_next = __ldg(&P.zt[lp + P.tpr]);
    int j0;
    float fr, rx;
    node_position(S, zt, P.B2hi, P.B2lo, j0, fr, rx);
    const float wt = P.wscale * zt.z * rx;
    float2 v, u;
    node_value_pair<H>(P, X, W, j0, fr, v, u);
    if (lp == nzh) {
      Zs[nzh] = make_float2(0.5f * wt * (v.x + u.x), 0.5f * wt * (v.y + u.y));
    } else {
      Zs[lp] = make_float2(wt * v.x, wt * v.y);
      Zs[P.nz - lp] = make_float2(wt * u.x, wt * u.y);
    }
  }
}

// Fetch the next work item for the whole CTA (dynamic scheduling).
__device__ __forceinline__ int next_item(int* counter, int* s_item) {
  __syncthreads();
  if (threadIdx.x == 0) *s_item = atomicAdd(counter, 1);
  __syncthreads();
  return *s_item;
}

// ZF = false: writes the half image spectrum fhat[k][l'] (both lateral
// destinations k and -k); ZF = true: writes the row's own full depth spectrum
// F[row][l mod nz] (see gather_row_z).
// PAIRED: the launch holds problems in the paired layout (RowProblem::paired);
// compiled apart so that the kernel of plans without them keeps its registers.
template <int H, bool ZF, bool PAIRED = false>
__global__ void __launch_bounds__(1024) row_forward_kernel(RowLaunch L, WindowPoly W) {
  extern __shared__ float2 smem[];
  __shared__ int s_item;
  for (;;) {
    const int item = next_item(L.counter, &s_item);
    if (item >= L.nitems) break;
    const WorkItem wi = L.items[item];
    const RowProblem& P = L.problems[wi.problem];
    const int tpr = P.tpr, M = P.M;
    const int slot = threadIdx.x / tpr;
    const int lane = threadIdx.x - slot * tpr;
    const int row = wi.row0 + slot;
    const bool valid = row < P.rows;
    float2* X = smem + slot * P.slot;
    // first pass straight from the lateral spectrum row (rows past the end read row 0, unused)
    const int srow = valid ? row : 0;
    const bool paired = PAIRED && P.paired != 0;
    const float2* src = P.pt + (size_t)srow * (paired ? P.nt >> 1 : P.nt);
    const float2* src2 = P.pt + (size_t)(srow == 0 ? 0 : P.n2 - srow) * (P.nt >> 1);
    const bool r32 = first_pass32(M, P.mshift, P.nt);
    // (the layout is a template argument so that each path issues its loads
    // back to back)
    if (PAIRED && paired) {
      if (r32) fft_first_pass32_from_global<true>(X, M, P.nt, lane, tpr, src, P.prescale, src2);
      else fft_first_pass_from_global<true>(X, M, P.nt, lane, tpr, src, P.prescale, src2);
    } else {
      if (r32) fft_first_pass32_from_global<false>(X, M, P.nt, lane, tpr, src, P.prescale, src2);
      else fft_first_pass_from_global<false>(X, M, P.nt, lane, tpr, src, P.prescale, src2);
    }
    // (rotated twiddles only in radix-8 last passes: the register pressure of
    // the radix-2/4 ones costs this kernel more than the table loads)
    fft_rest<false, kLayoutFlatGhost, 8>(X, M, P.mshift, lane, tpr, L.tw, L.Mmax >> P.mshift, true, r32 ? 5 : 4);
    if (valid) {
      if (!ZF) gather_row<H>(P, W, X, row, lane);
      else gather_row_z<H>(P, W, X, P.fh + (size_t)row * P.nz, row, lane);
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint
// ---------------------------------------------------------------------------

// Adjoint of the node evaluation.  Windowed methods: the node record carries
// e^{+i pi nu} (the transpose of the node's phase) and the taps weigh
// w_t(fr).  Interpolation methods (H = 2 plans only): the phase belongs to the
// grid cell, e^{+i pi nu_j}, applied to each cell after the spread, and tap
// t = 1, 2 (cells j0, j0+1) weigh 1 - fr, fr (linear) or 1 on the nearer cell.
template <int H>
__device__ __forceinline__ float2 adj_node_phase(const RowProblem& P, int j0, float fr) {
  if constexpr (H == 2) {
    if (P.method >= PAI_METHOD_LINEAR) return make_float2(1.0f, 0.0f);
  }
  return node_phase(j0, fr, P.nt, P.M, P.nt_over_M);
}

__device__ __forceinline__ float interp_tap_weight(int method, int t, float fr) {
  if (method == PAI_METHOD_NEAREST) return (t == 1) ? (fr >= 0.5f ? 0.0f : 1.0f) : (t == 2 ? (fr >= 0.5f ? 1.0f : 0.0f) : 0.0f);
  return (t == 1) ? 1.0f - fr : (t == 2 ? fr : 0.0f);
}

__device__ __forceinline__ int floor_div(int a, int b) {  // b > 0
  return (a >= 0) ? a / b : -((-a + b - 1) / b);
}

// Adjoint of one row by node pairs spread by one warp (spread mode 3,
// windowed methods, row slots of one or two warps).
//
// Phase 1: pair i holds the node pair +-x of one depth index (l = i + 1, or
// j = i in forward-model mode), sorted by x: A[i] = (j0, fr, Q+) for the +x
// node (x = j0 + fr) and B[i] = Q- for the -x node, each Q the node's input
// value times the weight and the transpose of its phase, e^{+i pi nu} for +x
// and its conjugate for -x.  The -x node is taken as (-j0 - 1) + (1 - fr), as
// the forward gather takes it, so its tap q weighs w_{2H-1-q}(z), z = fr - 1/2:
// one evaluation of the tap-pair polynomials serves both nodes.
//
// Phase 2: the row slot's first warp spreads all pairs into the grid X, 32
// consecutive pairs at a time, one per lane (with a second warp in the slot,
// as for M = 1024, that warp waits: a private grid for it cost more in
// occupancy than it saved); pairs with equal j0 form a run (the list is
// sorted), and for each tap pair and each of the four contributions (taps p
// and 2H-1-p of +x and of -x) the run's terms are summed across its lanes
// (segmented shuffle sum, only when the 32 pairs hold a run) and the run's
// first lane adds the sum to its cell with a plain read-modify-write.  Within
// one such step distinct runs have distinct j0, hence distinct cells (the 32
// pairs span fewer than M - 2H cells, checked by the plan); a __syncwarp
// separates the steps.  Every cell therefore receives its terms in a fixed
// order: the result is bit-repeatable.
// Returns whether the row is a mirror row (non-ZF input, both destinations).
// ATOM (spread mode 4, rows of any number of warps): every warp of the slot
// spreads its share of the 32-pair chunks, each run's sum added with
// shared-memory atomics (the order of the additions into a cell varies).
template <int H, bool ZF, bool ATOM = false>
__device__ __forceinline__ bool adjoint_pairs(const RowProblem& P, const WindowPoly& W, int row, bool valid, int lane,
                                              float2* X, float4* A) {
  const int tpr = P.tpr, M = P.M, nt = P.nt, mask = M - 1;
  const int nzh = P.nz >> 1;
  float2* B = reinterpret_cast<float2*>(A + nzh + 1);
  bool mirror = true;
  int np = 0;
  if (valid) {
    const float2* Zs = P.fh + (size_t)row * P.nz;  // ZF: the row's depth spectrum Fbar[l mod nz]
    if (ZF && P.qmode) {
      // forward model: pair j (j = 0..nz/2) carries c_j / 2 on both nodes,
      // c_j = F[j] + F[-j] (F[0], F[nz/2] alone); wscale holds 1 / (2 n_lat nz)
      const float2 S = P.rowS[row];
      np = nzh + 1;
      for (int j = lane; j <= nzh; j += tpr) {
        const float4 zt = __ldg(&P.zt[j]);
        int j0;
        float fr, rx;
        node_position(S, zt, P.B2hi, P.B2lo, j0, fr, rx);
        float2 y = Zs[j];
        if (j > 0 && j < nzh) y = cadd(y, Zs[P.nz - j]);
        const float2 pb = make_float2(P.wscale * y.x, P.wscale * y.y);
        const float2 ph = node_phase(j0, fr, nt, M, P.nt_over_M);
        const float2 qp = cmul(pb, ph), qn = cmul(pb, make_float2(ph.x, -ph.y));
        A[j] = make_float4(__int_as_float(j0), fr, qp.x, qp.y);
        B[j] = qn;
      }
    } else {
      RowGeom rg;
      const float2* in1 = nullptr;
      const float2* in2 = nullptr;
      if (ZF) {
        rg.S = P.rowS[row];
      } else {
        rg = row_geom(P, row);
        mirror = rg.mirror;
        in1 = P.fh + (size_t)rg.d1 * P.lz;
        in2 = P.fh + (size_t)rg.d2 * P.lz;
      }
      np = nzh;
      for (int i = lane; i < nzh; i += tpr) {
        const int lp = i + 1;
        const float4 zt = __ldg(&P.zt[lp]);
        int j0;
        float fr, rx;
        node_position(rg.S, zt, P.B2hi, P.B2lo, j0, fr, rx);
        const float wt = P.wscale * zt.z * rx;
        const float2 ph = node_phase(j0, fr, nt, M, P.nt_over_M);
        const float2 phc = make_float2(ph.x, -ph.y);
        float2 qp, qn;
        if (lp == nzh) {
          // Nyquist: both nodes carry half the l = -nz/2 input
          float2 y;
          if (ZF) {
            y = Zs[nzh];
          } else {
            y = in1[lp];
            if (mirror) {
              const float2 y2 = in2[lp];
              y.x += y2.x;
              y.y -= y2.y;
            }
          }
          const float2 pb = make_float2(0.5f * wt * y.x, 0.5f * wt * y.y);
          qp = cmul(pb, ph);
          qn = cmul(pb, phc);
        } else if (ZF) {
          const float2 y = Zs[lp], y2 = Zs[P.nz - lp];
          qp = cmul(make_float2(wt * y.x, wt * y.y), ph);
          qn = cmul(make_float2(wt * y2.x, wt * y2.y), phc);
        } else {
          const float2 y = in1[lp];
          qp = cmul(make_float2(2.0f * wt * y.x, 2.0f * wt * y.y), ph);
          if (mirror) {
            const float2 y2 = in2[lp];
            qn = cmul(make_float2(2.0f * wt * y2.x, -2.0f * wt * y2.y), phc);
          } else {
            qn = make_float2(0.f, 0.f);  // self-conjugate row: no -nu node below the Nyquist entry
          }
        }
        A[i] = make_float4(__int_as_float(j0), fr, qp.x, qp.y);
        B[i] = qn;
      }
    }
  }
  __syncthreads();  // pair lists complete (every row slot)
  // the row slot's first warp spreads every pair; a second warp (rows of
  // 64 threads) waits at the barrier below
  const int w = lane >> 5, l32 = lane & 31;
  float2* G = X;
  if (ATOM) {
    for (int g = lane; g < M; g += tpr) G[PADI(g)] = make_float2(0.f, 0.f);
    __syncthreads();  // the grid is zero before any warp adds to it
  } else if (w == 0) {
    for (int g = l32; g < M; g += 32) G[PADI(g)] = make_float2(0.f, 0.f);
    __syncwarp();
  }
  if (valid && (ATOM || w == 0)) {
    const unsigned full = 0xffffffffu;
    const int p1 = np;
    const int c_first = ATOM ? 32 * w : 0, c_step = ATOM ? tpr : 32;
    for (int c0 = c_first; c0 < p1; c0 += c_step) {
      const int i = c0 + l32;
      const bool act = i < p1;
      const float4 a = act ? A[i] : make_float4(0.f, 0.5f, 0.f, 0.f);
      const float2 b = act ? B[i] : make_float2(0.f, 0.f);
      const int j0 = __float_as_int(a.x);
      const int prev = __shfl_up_sync(full, j0, 1);
      const bool head = act && (l32 == 0 || prev != j0);
      const unsigned heads = __ballot_sync(full, head);
      const unsigned actm = __ballot_sync(full, act);
      // last lane of this lane's run
      const unsigned later = heads & (0xfffffffeu << l32);
      const int last = later ? __ffs(later) - 2 : 31 - __clz(actm);
      const int span = head ? last - l32 + 1 : 0;
      const int maxrun = __reduce_max_sync(full, (unsigned)span);
      const float2 qp = make_float2(a.z, a.w);
      const float z = a.y - 0.5f, z2 = z * z;
      const int cp0 = j0 - H + 1;  // cell of tap 0 of +x
      const int cn0 = -j0 - H;     // cell of tap 0 of -x
#pragma unroll
      for (int p = 0; p < H; ++p) {
        float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
        for (int e = kHalfCoef - 2; e >= 0; --e) {
          E = fmaf(E, z2, W.ce[p][e]);
          O = fmaf(O, z2, W.co[p][e]);
        }
        const float wl = fmaf(z, O, E), wh = fmaf(-z, O, E);
        // taps p and 2H-1-p of +x (weights wl, wh); of -x (wh, wl)
        float2 c[4] = {mul2(make_float2(wl, wl), qp), mul2(make_float2(wh, wh), qp), mul2(make_float2(wh, wh), b),
                       mul2(make_float2(wl, wl), b)};
        if (maxrun > 1) {
          for (int d = 1; d < maxrun; d <<= 1) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
              const float tx = __shfl_down_sync(full, c[k].x, d);
              const float ty = __shfl_down_sync(full, c[k].y, d);
              if (l32 + d <= last) {
                c[k].x += tx;
                c[k].y += ty;
              }
            }
          }
        }
        const int cell[4] = {cp0 + p, cp0 + 2 * H - 1 - p, cn0 + p, cn0 + 2 * H - 1 - p};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          if (head) {
            float2* q = G + PADI(cell[k] & mask);
            if (ATOM) {
              atomicAdd(&q->x, c[k].x);
              atomicAdd(&q->y, c[k].y);
            } else {
              *q = cadd(*q, c[k]);
            }
          }
          if (!ATOM) __syncwarp();
        }
      }
    }
  }
  __syncthreads();  // the grid is complete
  return mirror;
}

// The adjoint row kernel with the pair spread (spread mode 3), a kernel of its
// own so that its register allocation does not carry the other schemes.
template <int H, bool ZF, bool ATOM>
__global__ void __launch_bounds__(1024) row_adjoint_pairs_kernel(RowLaunch L, WindowPoly W) {
  extern __shared__ float2 smem[];
  __shared__ int s_item;
  float4* nodes_all = reinterpret_cast<float4*>(smem + L.fft_region);
  for (;;) {
    const int item = next_item(L.counter, &s_item);
    if (item >= L.nitems) break;
    const WorkItem wi = L.items[item];
    const RowProblem& P = L.problems[wi.problem];
    const int tpr = P.tpr, M = P.M, nt = P.nt;
    const int slot = threadIdx.x / tpr;
    const int lane = threadIdx.x - slot * tpr;
    const int row = wi.row0 + slot;
    const bool valid = row < P.rows;
    float2* X = smem + slot * P.slot;
    float4* N = nodes_all + slot * (P.nz + 2);
    const bool mirror = adjoint_pairs<H, ZF, ATOM>(P, W, row, valid, lane, X, N);
    const float scale = (valid && !ZF && mirror) ? 0.5f : 1.0f;
    float2* dst = const_cast<float2*>(P.pt) + (size_t)(valid ? row : 0) * nt;
    fft_inverse_crop(X, M, P.mshift, nt, lane, tpr, L.tw, L.Mmax >> P.mshift, dst, P.prescale, scale, valid);
  }
}

// ZF = false: input is the half image spectrum (image R2C over all axes) with
// both lateral destinations of a row; ZF = true: input is the row's own full
// depth spectrum Fbar[row][l mod nz].
template <int H, bool ZF>
__global__ void __launch_bounds__(1024) row_adjoint_kernel(RowLaunch L, WindowPoly W) {
  extern __shared__ float2 smem[];
  __shared__ int s_item;
  float4* nodes_all = reinterpret_cast<float4*>(smem + L.fft_region);
  for (;;) {
    const int item = next_item(L.counter, &s_item);
    if (item >= L.nitems) break;
    const WorkItem wi = L.items[item];
    const RowProblem& P = L.problems[wi.problem];
    const int tpr = P.tpr, M = P.M, nt = P.nt, mask = M - 1;
    const int slot = threadIdx.x / tpr;
    const int lane = threadIdx.x - slot * tpr;
    const int row = wi.row0 + slot;
    const bool valid = row < P.rows;
    float2* X = smem + slot * P.slot;
    float4* N = nodes_all + slot * (P.nz + 2);
    const int nzh = P.nz >> 1;
    RowGeom rg;
    int nneg = 1, nn = 0;
    // ZF: the row's depth spectrum Fbar[l mod nz] (depth FFT of the lateral R2C of the image)
    const float2* Zs = P.fh + (size_t)(valid ? row : 0) * P.nz;
    if (valid && ZF && P.qmode) {
      // Discrete forward model (the operator Q of Sec. 2 on a padded periodic
      // box): the row's temporal samples are sum_j c_j cos(2 pi nu_j n / nt)
      // over the depth frequencies j = 0..nz/2, nu_j >= 0 the frequency of
      // |K| (j = 0 included: its frequency is the lateral |K|), with
      // c_j = F[j] + F[-j] (F[0], F[nz/2] alone).  Each cosine is the node pair
      // +-nu_j with value c_j / 2 (wscale holds 1 / (2 n_lat nz)); the spread
      // below and the inverse FFT then sum the pairs like any adjoint row.
      rg.S = P.rowS[row];
      rg.mirror = true;
      nneg = nzh + 1;
      nn = 2 * nneg;
      for (int j = lane; j <= nzh; j += tpr) {
        const float4 zt = __ldg(&P.zt[j]);
        int j0p, j0;
        float frp, fr, rx;
        node_position(rg.S, zt, P.B2hi, P.B2lo, j0p, frp, rx);
        negate_node(j0p, frp, j0, fr);
        float2 y = Zs[j];
        if (j > 0 && j < nzh) {
          const float2 y2 = Zs[P.nz - j];
          y.x += y2.x;
          y.y += y2.y;
        }
        const float2 pb = make_float2(P.wscale * y.x, P.wscale * y.y);
        const float2 qp = cmul(pb, node_phase(j0p, frp, nt, M, P.nt_over_M));
        const float2 qn = cmul(pb, node_phase(j0, fr, nt, M, P.nt_over_M));
        N[nneg + j] = make_float4(__int_as_float(j0p), frp, qp.x, qp.y);
        N[nneg - 1 - j] = make_float4(__int_as_float(j0), fr, qn.x, qn.y);
      }
    } else if (valid && ZF) {
      rg.S = P.rowS[row];
      rg.mirror = true;
      nneg = nzh;
      nn = nneg + nzh;
      const int nA = P.nz - 1;
      for (int i = lane; i < nA; i += tpr) {
        int lp;
        bool neg, nyq;
        node_task(i, nzh, nA, lp, neg, nyq);
        const float4 zt = __ldg(&P.zt[lp]);
        int j0p, j0;
        float frp, fr, rx;
        node_position(rg.S, zt, P.B2hi, P.B2lo, j0p, frp, rx);
        const float wt = P.wscale * zt.z * rx;
        negate_node(j0p, frp, j0, fr);
        if (nyq) {
          const float2 y = Zs[nzh];
          const float2 pb = make_float2(0.5f * wt * y.x, 0.5f * wt * y.y);
          const float2 qp = cmul(pb, adj_node_phase<H>(P, j0p, frp));
          const float2 qn = cmul(pb, adj_node_phase<H>(P, j0, fr));
          N[nneg + nzh - 1] = make_float4(__int_as_float(j0p), frp, qp.x, qp.y);
          N[0] = make_float4(__int_as_float(j0), fr, qn.x, qn.y);
        } else if (!neg) {
          const float2 y = Zs[lp];
          const float2 q = cmul(make_float2(wt * y.x, wt * y.y), adj_node_phase<H>(P, j0p, frp));
          N[nneg + lp - 1] = make_float4(__int_as_float(j0p), frp, q.x, q.y);
        } else {
          const float2 y = Zs[P.nz - lp];
          const float2 q = cmul(make_float2(wt * y.x, wt * y.y), adj_node_phase<H>(P, j0, fr));
          N[nzh - lp] = make_float4(__int_as_float(j0), fr, q.x, q.y);
        }
      }
    }
    if (valid && !ZF) {
      rg = row_geom(P, row);
      nneg = rg.mirror ? nzh : 1;
      nn = nneg + nzh;
      // phase 1: node values Q = e^{+i pi nu} * Pbar, stored sorted by position
      const int nA = rg.mirror ? (P.nz - 1) : nzh;
      const float2* in1 = P.fh + (size_t)rg.d1 * P.lz;
      const float2* in2 = P.fh + (size_t)rg.d2 * P.lz;
      for (int i = lane; i < nA; i += tpr) {
        int lp;
        bool neg, nyq;
        node_task(i, nzh, nA, lp, neg, nyq);
        const float4 zt = __ldg(&P.zt[lp]);
        int j0p, j0;
        float frp, fr, rx;
        node_position(rg.S, zt, P.B2hi, P.B2lo, j0p, frp, rx);
        const float wt = P.wscale * zt.z * rx;
        negate_node(j0p, frp, j0, fr);
        if (nyq) {
          float2 y = in1[lp];
          if (rg.mirror) {
            const float2 y2 = in2[lp];
            y.x += y2.x;
            y.y -= y2.y;
          }
          const float2 pb = make_float2(0.5f * wt * y.x, 0.5f * wt * y.y);
          const float2 php = adj_node_phase<H>(P, j0p, frp);
          const float2 phn = adj_node_phase<H>(P, j0, fr);
          const float2 qp = cmul(pb, php), qn = cmul(pb, phn);
          N[nneg + nzh - 1] = make_float4(__int_as_float(j0p), frp, qp.x, qp.y);
          N[0] = make_float4(__int_as_float(j0), fr, qn.x, qn.y);
        } else if (!neg) {
          const float2 y = in1[lp];
          const float2 pb = make_float2(2.0f * wt * y.x, 2.0f * wt * y.y);
          const float2 q = cmul(pb, adj_node_phase<H>(P, j0p, frp));
          N[nneg + lp - 1] = make_float4(__int_as_float(j0p), frp, q.x, q.y);
        } else {
          const float2 y = in2[lp];
          const float2 pb = make_float2(2.0f * wt * y.x, -2.0f * wt * y.y);
          const float2 q = cmul(pb, adj_node_phase<H>(P, j0, fr));
          N[nzh - lp] = make_float4(__int_as_float(j0), fr, q.x, q.y);
        }
      }
    }
    __syncthreads();
    // phase 2: the spread (the transpose of the gather).  Node k adds
    // w_t(fr_k) Q_k to grid cell j0_k + t - H + 1 (mod M), t = 0..2H-1, by one
    // of three schemes (the plan times them and keeps the fastest; the tap
    // phases are also the deterministic choice).  Tap phases: nodes are taken in chunks of at most one node per thread that never mix
    // the two signs (-nu and +nu lists).  Nodes with equal j0 form a run (the
    // list is sorted); for each tap t in turn the head of every run evaluates
    // the tap weight of each of its nodes (tap index uniform over the CTA, so
    // the polynomial coefficients stay constant-bank operands) and adds the
    // run's sum to its cell.  Taps run in the order 0, 2H-1, 1, 2H-2, ... so a
    // tap and its mirror share one evaluation of the pair polynomials.  Within
    // a chunk distinct runs have distinct j0 and the chunk spans fewer than
    // M - 2H cells, so in one tap phase no two heads write the same cell; a
    // barrier separates the tap phases.  Every cell receives its terms in a
    // fixed order (chunk, tap, node): deterministic, no atomics.
    if (L.spread_mode == 1) {
      // shared-memory atomics: every node adds its 2H taps straight into the
      // grid, no tap phases (summation order, hence the last bits, may vary
      // from run to run)
      const bool interp = H == 2 && P.method >= PAI_METHOD_LINEAR;
      for (int g = lane; g < M; g += tpr) X[PADI(g)] = make_float2(0.f, 0.f);
      __syncthreads();
      for (int i = lane; i < nn; i += tpr) {
        const float4 nd = N[i];
        const int j0 = __float_as_int(nd.x);
        const float z = nd.y - 0.5f, z2 = z * z;
#pragma unroll
        for (int p = 0; p < H; ++p) {
          float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
          for (int e = kHalfCoef - 2; e >= 0; --e) {
            E = fmaf(E, z2, W.ce[p][e]);
            O = fmaf(O, z2, W.co[p][e]);
          }
          float wl = fmaf(z, O, E), wh = fmaf(-z, O, E);
          if constexpr (H == 2) {
            if (interp) {
              wl = interp_tap_weight(P.method, p, nd.y);
              wh = interp_tap_weight(P.method, 2 * H - 1 - p, nd.y);
            }
          }
          float2* cl = X + PADI((j0 + p - H + 1) & mask);
          float2* ch = X + PADI((j0 + H - p) & mask);
          atomicAdd(&cl->x, wl * nd.z);
          atomicAdd(&cl->y, wl * nd.w);
          atomicAdd(&ch->x, wh * nd.z);
          atomicAdd(&ch->y, wh * nd.w);
        }
      }
      __syncthreads();  // every node's taps are in the grid
    } else if (L.spread_mode == 2) {
      // shared-memory atomics per run: the first node of each run of equal j0
      // sums the run's weighted terms for every tap and adds each sum with one
      // atomic, so clusters of nodes on few cells cost few atomics
      const bool interp = H == 2 && P.method >= PAI_METHOD_LINEAR;
      for (int g = lane; g < M; g += tpr) X[PADI(g)] = make_float2(0.f, 0.f);
      __syncthreads();
      for (int i = lane; i < nn; i += tpr) {
        const int j0 = __float_as_int(N[i].x);
        if (i > 0 && __float_as_int(N[i - 1].x) == j0) continue;  // not the first node of its run
        int run = 1;
        while (i + run < nn && __float_as_int(N[i + run].x) == j0) ++run;
#pragma unroll
        for (int p = 0; p < H; ++p) {
          float lx = 0.f, ly = 0.f, hx = 0.f, hy = 0.f;  // taps p and 2H-1-p
          for (int r = 0; r < run; ++r) {
            const float4 nd = N[i + r];
            const float z = nd.y - 0.5f, z2 = z * z;
            float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
            for (int e = kHalfCoef - 2; e >= 0; --e) {
              E = fmaf(E, z2, W.ce[p][e]);
              O = fmaf(O, z2, W.co[p][e]);
            }
            float wl = fmaf(z, O, E), wh = fmaf(-z, O, E);
            if constexpr (H == 2) {
              if (interp) {
                wl = interp_tap_weight(P.method, p, nd.y);
                wh = interp_tap_weight(P.method, 2 * H - 1 - p, nd.y);
              }
            }
            lx = fmaf(wl, nd.z, lx);
            ly = fmaf(wl, nd.w, ly);
            hx = fmaf(wh, nd.z, hx);
            hy = fmaf(wh, nd.w, hy);
          }
          float2* cl = X + PADI((j0 + p - H + 1) & mask);
          float2* ch = X + PADI((j0 + H - p) & mask);
          atomicAdd(&cl->x, lx);
          atomicAdd(&cl->y, ly);
          atomicAdd(&ch->x, hx);
          atomicAdd(&ch->y, hy);
        }
      }
      __syncthreads();  // every run's taps are in the grid
    } else {
      const int CH = L.chunk;  // <= tpr
      const bool interp = H == 2 && P.method >= PAI_METHOD_LINEAR;
      for (int g = lane; g < M; g += tpr) X[PADI(g)] = make_float2(0.f, 0.f);
      const int list_max = (P.nz >> 1) + (P.qmode ? 1 : 0);  // nodes per sign list, at most
      const int half_chunks = (list_max + CH - 1) / CH;         // uniform over the CTA's slots
      for (int c = 0; c < 2 * half_chunks; ++c) {
        const bool pos = c >= half_chunks;
        const int first = pos ? nneg : 0;
        const int count = pos ? nn - nneg : nneg;
        const int c0 = first + (pos ? c - half_chunks : c) * CH;
        const int cn = valid ? max(0, min(CH, first + count - c0)) : 0;
        int j0 = 0, run = 0;  // run length if this thread's node heads a run, else 0
        if (lane < cn) {
          j0 = __float_as_int(N[c0 + lane].x);
          if (lane == 0 || __float_as_int(N[c0 + lane - 1].x) != j0) {
            run = 1;
            while (lane + run < cn && __float_as_int(N[c0 + lane + run].x) == j0) ++run;
          }
        }
        // the head's own node stays in registers for all taps; its polynomial
        // pair (E_p, O_p) serves tap p and its mirror 2H-1-p, which run in
        // consecutive phases
        const float4 nd0 = run > 0 ? N[c0 + lane] : make_float4(0.f, 0.f, 0.f, 0.f);
        const float z0 = nd0.y - 0.5f, z0sq = z0 * z0;
        __syncthreads();  // previous chunk's writes (or the zeroing) complete
#pragma unroll
        for (int p = 0; p < H; ++p) {
          float E0 = W.ce[p][kHalfCoef - 1], O0 = W.co[p][kHalfCoef - 1];
#pragma unroll
          for (int e = kHalfCoef - 2; e >= 0; --e) {
            E0 = fmaf(E0, z0sq, W.ce[p][e]);
            O0 = fmaf(O0, z0sq, W.co[p][e]);
          }
#pragma unroll
          for (int side = 0; side < 2; ++side) {
            // tap t = p (side 0) or 2H-1-p (side 1): w(z) = E_p(z^2) +- z O_p(z^2), z = fr - 1/2
            const int t = side == 0 ? p : 2 * H - 1 - p;
            if (run > 0) {
              float w0 = side == 0 ? fmaf(z0, O0, E0) : fmaf(-z0, O0, E0);
              if constexpr (H == 2) {
                if (interp) w0 = interp_tap_weight(P.method, t, nd0.y);
              }
              float sx = w0 * nd0.z, sy = w0 * nd0.w;
              for (int r = 1; r < run; ++r) {
                const float4 nd = N[c0 + lane + r];
                const float z = side == 0 ? nd.y - 0.5f : 0.5f - nd.y;
                const float z2 = z * z;
                float E = W.ce[p][kHalfCoef - 1], O = W.co[p][kHalfCoef - 1];
#pragma unroll
                for (int e = kHalfCoef - 2; e >= 0; --e) {
                  E = fmaf(E, z2, W.ce[p][e]);
                  O = fmaf(O, z2, W.co[p][e]);
                }
                float w = fmaf(z, O, E);
                if constexpr (H == 2) {
                  if (interp) w = interp_tap_weight(P.method, t, nd.y);
                }
                sx = fmaf(w, nd.z, sx);
                sy = fmaf(w, nd.w, sy);
              }
              const int gi = PADI((j0 + t - H + 1) & mask);
              float2 x = X[gi];
              x.x += sx;
              x.y += sy;
              X[gi] = x;
            }
            __syncthreads();
          }
        }
      }
    }
    if constexpr (H == 2) {
      // interpolation methods: the grid cells' phases e^{+i pi nu_j}
      if (valid && P.method >= PAI_METHOD_LINEAR)
        for (int g = lane; g < M; g += tpr) X[PADI(g)] = cmul(X[PADI(g)], node_phase(g, 0.0f, nt, M, P.nt_over_M));
    }
    __syncthreads();
    const float scale = (valid && !ZF && rg.mirror) ? 0.5f : 1.0f;
    float2* dst = const_cast<float2*>(P.pt) + (size_t)(valid ? row : 0) * nt;
    fft_inverse_crop(X, M, P.mshift, nt, lane, tpr, L.tw, L.Mmax >> P.mshift, dst, P.prescale, scale, valid);
  }
}

}  // namespace pai
