// Batched mixed-radix FFT stages in shared memory (radix 2, 3, 4, 5).
//
// The kinetic term of Eq. localproblem is applied spectrally (Sec. II.B,
// operation 1: "applying the Laplacian operator via the FFT").  Transforms
// here are Stockham autosort stages: each butterfly reads R inputs n/R apart,
// applies the twiddles e^{-+2 pi i r k / (Ns R)}, does a length-R DFT and
// writes R outputs Ns apart, so the result is in natural order after the
// last stage.  Twiddles come from a host-computed FP64 table of
// e^{-2 pi i t / n}; the inverse uses their conjugates.  Lines live in shared
// memory at base + line * ls + pos * es, so the same stage code transforms
// rows (es = 1) and columns (ls = 1) of a plane.
#pragma once

#include "common.cuh"

namespace dgdft {

template <class C, int R, bool INV>
__device__ __forceinline__ void small_dft(C* v, const C* tw, int n) {
  if (R == 2) {
    C a = v[0], b = v[1];
    v[0] = cadd(a, b);
    v[1] = csub(a, b);
  } else if (R == 4) {
    C a0 = cadd(v[0], v[2]), a1 = csub(v[0], v[2]);
    C a2 = cadd(v[1], v[3]), a3 = csub(v[1], v[3]);
    // forward: multiply a3 by -i; inverse: by +i
    C a3r = INV ? cmake<C>(-a3.y, a3.x) : cmake<C>(a3.y, -a3.x);
    v[0] = cadd(a0, a2);
    v[2] = csub(a0, a2);
    v[1] = cadd(a1, a3r);
    v[3] = csub(a1, a3r);
  } else {
    // generic length-R DFT with roots taken from the twiddle table
    C root[R];
#pragma unroll
    for (int s = 0; s < R; ++s) {
      C w = tw[s * (n / R)];
      root[s] = INV ? cconj(w) : w;
    }
    C out[R];
#pragma unroll
    for (int q = 0; q < R; ++q) {
      C acc = v[0];
#pragma unroll
      for (int r = 1; r < R; ++r) acc = cadd(acc, cmul(v[r], root[(r * q) % R]));
      out[q] = acc;
    }
#pragma unroll
    for (int q = 0; q < R; ++q) v[q] = out[q];
  }
}

// floor(a / d) for 0 <= a < 2^16, 2 <= d < 2^16 by one high multiply: with
// M = ceil(2^32 / d), a M / 2^32 = a / d + a (M d - 2^32) / (d 2^32) and the
// second term is below 1 / d, so the integer part is exact.  M does not fit
// 32 bits for d = 1, which is marked by M = 0 and handled apart.
__device__ __forceinline__ unsigned div_magic(unsigned d) { return d > 1u ? 0xFFFFFFFFu / d + 1u : 0u; }
__device__ __forceinline__ int udiv_small(int a, unsigned magic) {
  return magic ? (int)__umulhi((unsigned)a, magic) : a;
}

template <class C, int R, bool INV>
__device__ __forceinline__ void stage_radix(const C* __restrict__ in, C* __restrict__ out, int n,
                                            int Ns, int nlines, int ls, int es, const C* tw) {
  const int nb = n / R;
  const int total = nlines * nb;
  const int tstep = n / (Ns * R);
  const unsigned mag_nb = div_magic(nb), mag_ns = div_magic(Ns);
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int l = udiv_small(b, mag_nb);
    const int j = b - l * nb;
    const int jq = udiv_small(j, mag_ns);
    const int k = j - jq * Ns;
    C v[R];
    const C* src = in + l * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * es];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * tstep];
        v[r] = cmul(v[r], INV ? cconj(w) : w);
      }
    }
    small_dft<C, R, INV>(v, tw, n);
    const int idxD = jq * Ns * R + k;
    C* dst = out + l * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(idxD + r * Ns) * es] = v[r];
  }
}

// Compile-time variant for a line length N known when the kernel is built:
// the same radix order as the host plan (4s, then 2s, 3s, 5s), every loop
// bound, stride and twiddle step a constant.
__host__ __device__ constexpr int ct_nstage(int n) {
  int s = 0;
  const int rad[4] = {4, 2, 3, 5};
  for (int q = 0; q < 4; ++q)
    while (n % rad[q] == 0) {
      n /= rad[q];
      ++s;
    }
  return s;
}
__host__ __device__ constexpr int ct_radix(int n, int stage) {
  int s = 0;
  const int rad[4] = {4, 2, 3, 5};
  for (int q = 0; q < 4; ++q)
    while (n % rad[q] == 0) {
      if (s == stage) return rad[q];
      n /= rad[q];
      ++s;
    }
  return 1;
}

template <class C, int R, bool INV, int N, int NS>
__device__ __forceinline__ void stage_radix_ct(const C* __restrict__ in, C* __restrict__ out, int nlines, int ls,
                                               int es, const C* tw) {
  constexpr int nb = N / R;
  constexpr int tstep = N / (NS * R);
  const int total = nlines * nb;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int l = b / nb;
    const int j = b - l * nb;
    const int jq = j / NS;
    const int k = j - jq * NS;
    C v[R];
    const C* src = in + l * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[(j + r * nb) * es];
    if (NS > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        C w = tw[r * k * tstep];
        v[r] = cmul(v[r], INV ? cconj(w) : w);
      }
    }
    small_dft<C, R, INV>(v, tw, N);
    const int idxD = jq * NS * R + k;
    C* dst = out + l * ls;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[(idxD + r * NS) * es] = v[r];
  }
}

template <class C, bool INV, int N, int S, int NS>
__device__ __forceinline__ int fft_ct_stages(C* buf0, C* buf1, int cur, int nlines, int ls, int es, const C* tw) {
  if constexpr (S >= ct_nstage(N)) {
    return cur;
  } else {
    constexpr int R = ct_radix(N, S);
    stage_radix_ct<C, R, INV, N, NS>(cur ? buf1 : buf0, cur ? buf0 : buf1, nlines, ls, es, tw);
    __syncthreads();
    return fft_ct_stages<C, INV, N, S + 1, NS * R>(buf0, buf1, cur ^ 1, nlines, ls, es, tw);
  }
}

// N > 0: the compile-time transform; N == 0: the plan's runtime transform.
template <class C, bool INV, int N>
__device__ __forceinline__ int fft_lines_n(C* buf0, C* buf1, int cur, const FftPlan& plan, int nlines, int ls,
                                           int es, const C* tw);

// Full transform of nlines lines; ping-pongs between bufs[0] and bufs[1]
// starting from bufs[cur].  Returns the index of the buffer holding the result.
// Must be called by every thread of the block.
template <class C, bool INV>
__device__ int fft_lines(C* buf0, C* buf1, int cur, const FftPlan& plan, int nlines, int ls,
                         int es, const C* tw) {
  int Ns = 1;
  for (int s = 0; s < plan.nstage; ++s) {
    const int R = plan.radix[s];
    C* in = cur ? buf1 : buf0;
    C* out = cur ? buf0 : buf1;
    switch (R) {
      case 2: stage_radix<C, 2, INV>(in, out, plan.n, Ns, nlines, ls, es, tw); break;
      case 3: stage_radix<C, 3, INV>(in, out, plan.n, Ns, nlines, ls, es, tw); break;
      case 4: stage_radix<C, 4, INV>(in, out, plan.n, Ns, nlines, ls, es, tw); break;
      default: stage_radix<C, 5, INV>(in, out, plan.n, Ns, nlines, ls, es, tw); break;
    }
    __syncthreads();
    Ns *= R;
    cur ^= 1;
  }
  return cur;
}

template <class C, bool INV, int N>
__device__ __forceinline__ int fft_lines_n(C* buf0, C* buf1, int cur, const FftPlan& plan, int nlines, int ls,
                                           int es, const C* tw) {
  if constexpr (N > 0)
    return fft_ct_stages<C, INV, N, 0, 1>(buf0, buf1, cur, nlines, ls, es, tw);
  else
    return fft_lines<C, INV>(buf0, buf1, cur, plan, nlines, ls, es, tw);
}

}  // namespace dgdft
