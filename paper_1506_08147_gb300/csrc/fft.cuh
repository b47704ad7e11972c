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

// floor(a / d) for 0 <= a < 2^22 from a rounded reciprocal: (a + 0.5) / d
// lies at least 0.5 / d from an integer, far beyond the FP32 rounding of
// the product, so truncation gives the exact quotient.
__device__ __forceinline__ int fdiv_small(int a, float inv_d) {
  return __float2int_rz(((float)a + 0.5f) * inv_d);
}

template <class C, int R, bool INV>
__device__ __forceinline__ void stage_radix(const C* __restrict__ in, C* __restrict__ out, int n,
                                            int Ns, int nlines, int ls, int es, const C* tw) {
  const int nb = n / R;
  const int total = nlines * nb;
  const int tstep = n / (Ns * R);
  const float inv_nb = 1.0f / (float)nb, inv_ns = 1.0f / (float)Ns;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int l = fdiv_small(b, inv_nb);
    const int j = b - l * nb;
    const int jq = fdiv_small(j, inv_ns);
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

}  // namespace dgdft
