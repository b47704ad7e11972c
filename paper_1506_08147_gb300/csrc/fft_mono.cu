// H apply and Teter preconditioner for the monolayer grids (48 x 64 x 40 and
// 48 x 64 x 48), FP32 stage.
//
// Sec. II.B, operation 1 (the Laplacian applied via the FFT) and operation 5
// (the Teter preconditioner), the same three passes over HBM as the general
// kernels, but with the short transforms held in registers instead of
// shared-memory stages separated by barriers:
//   fwd : one z-plane of one vector per CTA (64 threads, 14.4 KB of shared
//         memory, 12 CTAs per SM, so that the load, transform and store
//         phases of different CTAs overlap); each thread owns one x row
//         (48 reals -> 24-point complex FFT in registers -> r2c split to 25
//         complex), then the 64-point y lines as an 8 x 8 four-step transform
//         inside a warp (8 lanes per line, __syncwarp only);
//   z   : one thread per (kx, y) column: 40- or 48-point FFT in registers,
//         the kinetic symbol (or the Teter factor, or the sphere-cutoff
//         mask), inverse FFT;
//   inv : the inverse y lines, then per row the c2r recombination and the
//         24-point inverse in registers, then the epilogue (Kleinman-Bylander
//         scatter, (V - sigma) psi) on the plane in shared memory.
// The half spectrum between the passes is ordered [z][kx][y] (the general
// kernels order it [z][y][kx]; the two sets never share a spectrum).
// Twiddles e^{-2 pi i t / n} come from host-computed FP64 tables rounded to
// FP32, in constant memory (every index is a compile-time constant after
// unrolling) or, for the lane-dependent four-step twiddles, shared memory.
#include <cmath>

#include "fft.cuh"
#include "internal.h"

namespace dgdft {

namespace {

constexpr int MX = 48, MH = 24, MXH = 25, MY = 64;
constexpr int MPL = 1;                  // z-planes per CTA (nz % MPL == 0)
constexpr int MLINE = 72;               // padded y line: position y + y / 8
constexpr int MROW = 52;                // padded real row (48 + 4): conflict-free float4 rows
constexpr int MPLANE = MX * MY;         // 3072 reals per plane
constexpr int MSPEC = MXH * MY;         // 1600 complex per plane of the half spectrum
constexpr int MTHREADS = 64 * MPL;      // one thread per row of the CTA's planes
constexpr int MCTAS = 12 / MPL;         // CTAs per SM (shared memory, registers)
constexpr int ZTHREADS = 160;           // z pass: 10 CTAs x 160 = 1600 columns
constexpr size_t MSMEM = sizeof(float2) * MPL * MXH * MLINE;  // 14,400 B per plane (the real rows alias it)

__constant__ float2 c_w48[48];
__constant__ float2 c_w64[64];
__constant__ float2 c_w40[40];

// e^{-+2 pi i t / N} for the register transforms (t < N, t a constant).
template <int N, bool INV>
__device__ __forceinline__ float2 twr(int t) {
  float2 w;
  if constexpr (N == 48) w = c_w48[t];
  else if constexpr (N == 24) w = c_w48[2 * t];
  else if constexpr (N == 64) w = c_w64[t];
  else if constexpr (N == 8) w = c_w64[8 * t];
  else w = c_w40[t];
  if (INV) w.y = -w.y;
  return w;
}

// Length-R DFT in registers (forward e^{-2 pi i r q / R}; INV: conjugate roots).
template <int R, bool INV>
__device__ __forceinline__ void rdft(float2 (&t)[R]) {
  if constexpr (R == 2) {
    const float2 a = t[0], b = t[1];
    t[0] = cadd(a, b);
    t[1] = csub(a, b);
  } else if constexpr (R == 4) {
    const float2 a0 = cadd(t[0], t[2]), a1 = csub(t[0], t[2]);
    const float2 a2 = cadd(t[1], t[3]), a3 = csub(t[1], t[3]);
    const float2 a3r = INV ? make_float2(-a3.y, a3.x) : make_float2(a3.y, -a3.x);  // -+i a3
    t[0] = cadd(a0, a2);
    t[2] = csub(a0, a2);
    t[1] = cadd(a1, a3r);
    t[3] = csub(a1, a3r);
  } else if constexpr (R == 3) {
    // X1,2 = t0 - (t1 + t2) / 2 -+ i (sqrt 3 / 2)(t1 - t2)
    constexpr float s3 = 0.86602540378443865f;
    const float2 s = cadd(t[1], t[2]), d = csub(t[1], t[2]);
    const float2 m = make_float2(t[0].x - 0.5f * s.x, t[0].y - 0.5f * s.y);
    const float2 n = INV ? make_float2(-s3 * d.y, s3 * d.x) : make_float2(s3 * d.y, -s3 * d.x);
    t[0] = cadd(t[0], s);
    t[1] = cadd(m, n);
    t[2] = csub(m, n);
  } else {
    static_assert(R == 5, "radix");
    // c1,2 = cos(2 pi / 5), cos(4 pi / 5); s1,2 = sin(2 pi / 5), sin(4 pi / 5)
    constexpr float c1 = 0.30901699437494742f, c2 = -0.80901699437494742f;
    constexpr float s1 = 0.95105651629515357f, s2 = 0.58778525229247313f;
    const float2 a1 = cadd(t[1], t[4]), b1 = csub(t[1], t[4]);
    const float2 a2 = cadd(t[2], t[3]), b2 = csub(t[2], t[3]);
    const float2 m1 = make_float2(t[0].x + c1 * a1.x + c2 * a2.x, t[0].y + c1 * a1.y + c2 * a2.y);
    const float2 m2 = make_float2(t[0].x + c2 * a1.x + c1 * a2.x, t[0].y + c2 * a1.y + c1 * a2.y);
    const float2 n1 = make_float2(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y);
    const float2 n2 = make_float2(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y);
    // forward: X1 = m1 - i n1, X4 = m1 + i n1, X2 = m2 - i n2, X3 = m2 + i n2
    const float2 in1 = INV ? make_float2(-n1.y, n1.x) : make_float2(n1.y, -n1.x);
    const float2 in2 = INV ? make_float2(-n2.y, n2.x) : make_float2(n2.y, -n2.x);
    t[0] = make_float2(t[0].x + a1.x + a2.x, t[0].y + a1.y + a2.y);
    t[1] = cadd(m1, in1);
    t[4] = csub(m1, in1);
    t[2] = cadd(m2, in2);
    t[3] = csub(m2, in2);
  }
}

// Stockham stages in registers, radices in the order of ct_radix: stage S
// reads R inputs N/R apart, twiddles them by e^{-+2 pi i r k / (NS R)}, does
// the length-R DFT and writes R outputs NS apart (natural order at the end).
template <int N, int S, int NS, bool INV>
__device__ __forceinline__ void rstages(float2 (&v)[N]) {
  if constexpr (S < ct_nstage(N)) {
    constexpr int R = ct_radix(N, S);
    constexpr int NB = N / R;
    constexpr int TSTEP = N / (NS * R);
    float2 o[N];
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      const int jq = j / NS, k = j - (j / NS) * NS;
      float2 t[R];
#pragma unroll
      for (int r = 0; r < R; ++r) t[r] = v[j + r * NB];
      if (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r)
          if (r * k) t[r] = cmul(t[r], twr<N, INV>(r * k * TSTEP));
      }
      rdft<R, INV>(t);
#pragma unroll
      for (int r = 0; r < R; ++r) o[jq * NS * R + k + r * NS] = t[r];
    }
#pragma unroll
    for (int i = 0; i < N; ++i) v[i] = o[i];
    rstages<N, S + 1, NS * R, INV>(v);
  }
}

template <int N, bool INV>
__device__ __forceinline__ void rfft(float2 (&v)[N]) {
  rstages<N, 0, 1, INV>(v);
}

__device__ __forceinline__ bool live(const ElemDev<float>& e, int filt) {
  return e.state[ST_ACTIVE] != 0 && (filt == 0 || e.state[ST_TETER] != 0);
}

// The 64-point y transforms of the MPL x 25 lines of a CTA's planes, in place
// in the padded line layout.  Lane group g = lane / 8 of a warp takes one
// line, lane q = lane % 8 its points q + 8 i (four-step: an 8-point DFT over
// i, the twiddle w64^(q k1), an 8-point DFT over q).  Every thread calls it.
template <bool INV>
__device__ __forceinline__ void y_lines(float2* spec, const float2* w64s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, q = lane & 7;
  for (int base = warp * 4; base < MPL * MXH; base += (MTHREADS / 32) * 4) {
    const int li = base + (lane >> 3);
    const bool on = li < MPL * MXH;
    float2* L = spec + (size_t)(on ? li : 0) * MLINE;
    float2 a[8];
    if (on) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = L[q + 9 * i];  // point q + 8 i
      rfft<8, INV>(a);
#pragma unroll
      for (int k1 = 1; k1 < 8; ++k1) {
        float2 w = w64s[(q * k1) & 63];
        if (INV) w.y = -w.y;
        a[k1] = cmul(a[k1], w);
      }
#pragma unroll
      for (int k1 = 0; k1 < 8; ++k1) L[q + 9 * k1] = a[k1];  // point q + 8 k1
    }
    __syncwarp();
    if (on) {
#pragma unroll
      for (int i = 0; i < 8; ++i) a[i] = L[9 * q + i];  // point 8 q + i: B_i[k1 = q]
      rfft<8, INV>(a);
    }
    __syncwarp();
    if (on) {
#pragma unroll
      for (int k2 = 0; k2 < 8; ++k2) L[q + 9 * k2] = a[k2];  // point q + 8 k2
    }
    __syncwarp();
  }
}

__device__ __forceinline__ void load_w64(float2* w64s) {
  if (threadIdx.x < 64) w64s[threadIdx.x] = c_w64[threadIdx.x];
}

// Pass 1.  grid (nz / 4, columns, elements), 256 threads.
__global__ void __launch_bounds__(MTHREADS, MCTAS)
    mono_fwd_kernel(const ElemDev<float>* __restrict__ elems, BRef<float> src, int ncols, int filt, int nz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 w64s[64];
  const ElemDev<float>& e = elems[blockIdx.z];
  const int j = blockIdx.y, z0 = blockIdx.x * MPL;
  const int nc = ncols > 0 ? ncols : e.m;
  if (!live(e, filt) || j >= nc || e.nx != MX || e.ny != MY || e.nz != nz) return;
  float* rows = reinterpret_cast<float*>(smem_raw);
  float2* spec = reinterpret_cast<float2*>(smem_raw);
  load_w64(w64s);
  const float4* in4 = reinterpret_cast<const float4*>(resolve(e, src) + (size_t)j * e.ng + (size_t)z0 * MPLANE);
  for (int t = threadIdx.x; t < MPL * MPLANE / 4; t += MTHREADS) {
    const int row = t / 12, q = t - row * 12;
    *reinterpret_cast<float4*>(rows + row * MROW + 4 * q) = __ldg(in4 + t);
  }
  __syncthreads();
  // x: z_n = x_2n + i x_2n+1, 24-point FFT, split into the 25 outputs
  const int p = threadIdx.x >> 6, y = threadIdx.x & 63;
  float2 zr[MH];
  {
    const float4* r4 = reinterpret_cast<const float4*>(rows + threadIdx.x * MROW);
#pragma unroll
    for (int q = 0; q < 12; ++q) {
      const float4 v = r4[q];
      zr[2 * q] = make_float2(v.x, v.y);
      zr[2 * q + 1] = make_float2(v.z, v.w);
    }
  }
  rfft<MH, false>(zr);
  __syncthreads();  // the spectrum overwrites the rows
  {
    float2* col = spec + (size_t)p * MXH * MLINE + y + (y >> 3);
#pragma unroll
    for (int k = 0; k <= MH; ++k) {
      // X[k] = E[k] + e^{-2 pi i k / 48} O[k]
      const float2 zk = zr[k == MH ? 0 : k];
      const float2 zc = cconj(zr[k == 0 ? 0 : MH - k]);
      const float2 ev = cscale(cadd(zk, zc), 0.5f);
      const float2 df = csub(zk, zc);
      const float2 od = make_float2(0.5f * df.y, -0.5f * df.x);
      col[k * MLINE] = cadd(ev, cmul(c_w48[k], od));
    }
  }
  __syncthreads();
  y_lines<false>(spec, w64s);
  __syncthreads();
  float2* out = reinterpret_cast<float2*>(e.Z) + (size_t)j * e.nspec + (size_t)z0 * MSPEC;
  for (int t = threadIdx.x; t < MPL * MSPEC; t += MTHREADS) {
    const int pp = t / MSPEC, rem = t - pp * MSPEC;
    const int k = rem >> 6, yy = rem & 63;
    out[t] = spec[(size_t)(pp * MXH + k) * MLINE + yy + (yy >> 3)];
  }
}

// Pass 2.  grid (10, columns, elements), 160 threads: one (kx, y) column each.
template <int NZ, int MODE>
__global__ void __launch_bounds__(ZTHREADS)
    mono_z_kernel(const ElemDev<float>* __restrict__ elems, int ncols, const double* __restrict__ tkin_override,
                  int filt) {
  const ElemDev<float>& e = elems[blockIdx.z];
  const int j = blockIdx.y;
  const int nc = ncols > 0 ? ncols : e.m;
  if (!live(e, filt) || j >= nc || e.nx != MX || e.ny != MY || e.nz != NZ) return;
  const int c = blockIdx.x * ZTHREADS + threadIdx.x;  // < 1600
  const int kx = c >> 6, y = c & 63;
  float2* col = reinterpret_cast<float2*>(e.Z) + (size_t)j * e.nspec + c;
  float2 v[NZ];
#pragma unroll
  for (int z = 0; z < NZ; ++z) v[z] = col[(size_t)z * MSPEC];
  rfft<NZ, false>(v);
  const float gxy = e.gx2f[kx] + e.gy2f[y];
  const float scalef = (float)e.scale;
  const float ecutf = (float)e.ecut;  // mask of the sphere-cutoff set (FP32 decision)
  float inv_tk = 1.f;
  if (MODE == ZM_TETER) {
    // FP32 reciprocal: one FP64 division per thread costs ~16 FP64-pipe
    // cycles per instruction here
    const float tk = (float)(tkin_override ? tkin_override[j] : e.tkin[j]);
    inv_tk = 1.0f / fmaxf(tk, 1e-8f);
  }
#pragma unroll
  for (int z = 0; z < NZ; ++z) {
    const float g = gxy + e.gz2f[z];
    float f = g;
    if (MODE == ZM_TETER) {
      const float sv = g * inv_tk;
      const float num = 27.0f + sv * (18.0f + sv * (12.0f + sv * 8.0f));
      f = num / (num + 16.0f * sv * sv * sv * sv);
    } else if (MODE == ZM_MASK) {
      f = (g <= ecutf) ? 1.0f : 0.0f;
    }
    v[z] = cscale(v[z], f * scalef);
  }
  rfft<NZ, true>(v);
#pragma unroll
  for (int z = 0; z < NZ; ++z) col[(size_t)z * MSPEC] = v[z];
}

// Pass 3.  grid (nz / 4, columns, elements), 256 threads.
template <int MODE>
__global__ void __launch_bounds__(MTHREADS, MCTAS)
    mono_inv_kernel(const ElemDev<float>* __restrict__ elems, BRef<float> dst, BRef<float> xsrc, int ncols,
                    int filt, int nz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float2 w64s[64];
  const ElemDev<float>& e = elems[blockIdx.z];
  const int j = blockIdx.y, z0 = blockIdx.x * MPL;
  const int nc = ncols > 0 ? ncols : e.m;
  if (!live(e, filt) || j >= nc || e.nx != MX || e.ny != MY || e.nz != nz) return;
  float* rows = reinterpret_cast<float*>(smem_raw);
  float2* spec = reinterpret_cast<float2*>(smem_raw);
  load_w64(w64s);
  const float2* in = reinterpret_cast<const float2*>(e.Z) + (size_t)j * e.nspec + (size_t)z0 * MSPEC;
  for (int t = threadIdx.x; t < MPL * MSPEC; t += MTHREADS) {
    const int pp = t / MSPEC, rem = t - pp * MSPEC;
    const int k = rem >> 6, yy = rem & 63;
    spec[(size_t)(pp * MXH + k) * MLINE + yy + (yy >> 3)] = in[t];
  }
  __syncthreads();
  y_lines<true>(spec, w64s);
  __syncthreads();
  // x: recombine the half spectrum into E + i O, 24-point inverse
  const int p = threadIdx.x >> 6, y = threadIdx.x & 63;
  float2 zr[MH];
  {
    const float2* col = spec + (size_t)p * MXH * MLINE + y + (y >> 3);
    float2 X[MXH];
#pragma unroll
    for (int k = 0; k <= MH; ++k) X[k] = col[k * MLINE];
#pragma unroll
    for (int k = 0; k < MH; ++k) {
      const float2 xk = X[k], xc = cconj(X[MH - k]);
      const float2 ev = cscale(cadd(xk, xc), 0.5f);
      const float2 od = cmul(cscale(csub(xk, xc), 0.5f), cconj(c_w48[k]));
      zr[k] = make_float2(ev.x - od.y, ev.y + od.x);
    }
  }
  rfft<MH, true>(zr);
  __syncthreads();  // the rows overwrite the spectrum
  {
    float4* r4 = reinterpret_cast<float4*>(rows + threadIdx.x * MROW);
#pragma unroll
    for (int q = 0; q < 12; ++q)
      r4[q] = make_float4(zr[2 * q].x, zr[2 * q].y, zr[2 * q + 1].x, zr[2 * q + 1].y);
  }
  __syncthreads();
  const size_t off = (size_t)j * e.ng + (size_t)z0 * MPLANE;
  float4* out4 = reinterpret_cast<float4*>(resolve(e, dst) + off);
  if (MODE == XI_HAMILTONIAN) {
    if (e.n_sup > 0) {
      // Kleinman-Bylander scatter: each support point of the CTA's planes once.
      // The coefficients of column j go to the shared-memory tail past the
      // rows (free once the spectrum is consumed); each thread takes SU
      // points at a time and their nonzeros four at a time, so the loads of
      // different points are in flight together.
      constexpr int CTAIL = (int)(MSMEM / sizeof(float)) - MPL * MY * MROW;  // may be < 0: not staged
      constexpr int SU = 4;
      float* ctail = rows + MPL * MY * MROW;
      const float* cg = e.Ccoef + (size_t)j * e.n_proj;
      const bool staged = e.n_proj <= CTAIL;
      if (staged)
        for (int q = threadIdx.x; q < e.n_proj; q += MTHREADS) ctail[q] = cg[q];
      const float* cj = staged ? ctail : cg;
      const int sb = e.s_plane[z0], se = e.s_plane[z0 + MPL];
      int bnd[MPL > 1 ? MPL - 1 : 1];  // first support point of planes 1 .. MPL - 1
#pragma unroll
      for (int i = 0; i < MPL - 1; ++i) bnd[i] = e.s_plane[z0 + 1 + i];
      __syncthreads();
      for (int s0 = sb + threadIdx.x; s0 < se; s0 += SU * MTHREADS) {
        int qb[SU], qe[SU], o[SU];
        float acc[SU];
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          const int s = s0 + u * MTHREADS;
          const bool in = s < se;
          qb[u] = (in && !e.s_gv4) ? e.s_ptr[s] : 0;
          qe[u] = (in && !e.s_gv4) ? e.s_ptr[s + 1] : 0;
          o[u] = in ? e.s_off[s] : 0;
          acc[u] = 0.f;
        }
        if (e.s_gv4) {
          // at most 4 nonzeros per point, padded with zero weights
#pragma unroll
          for (int u = 0; u < SU; ++u) {
            const int s = s0 + u * MTHREADS;
            if (s < se) {
              const float4 g = __ldg(reinterpret_cast<const float4*>(e.s_gv4) + s);
              const int4 pj = __ldg(reinterpret_cast<const int4*>(e.s_proj4) + s);
              float a = g.x * cj[pj.x];
              a += g.y * cj[pj.y];
              a += g.z * cj[pj.z];
              a += g.w * cj[pj.w];
              acc[u] = a;
            }
          }
        } else {
          for (int k0 = 0;; k0 += 4) {
            bool more = false;
#pragma unroll
            for (int u = 0; u < SU; ++u) {
#pragma unroll
              for (int k = 0; k < 4; ++k) {
                const int q = qb[u] + k0 + k;
                if (q < qe[u]) acc[u] += e.s_gv[q] * cj[e.s_proj[q]];
              }
              more |= qb[u] + k0 + 4 < qe[u];
            }
            if (!more) break;
          }
        }
#pragma unroll
        for (int u = 0; u < SU; ++u) {
          const int s = s0 + u * MTHREADS;
          if (s < se) {
            int pz = 0;
#pragma unroll
            for (int i = 0; i < MPL - 1; ++i) pz += s >= bnd[i];
            const int yy = o[u] / MX, xx = o[u] - yy * MX;
            rows[(pz * MY + yy) * MROW + xx] += acc[u];
          }
        }
      }
      __syncthreads();
    }
    const float4* x4 = reinterpret_cast<const float4*>(resolve(e, xsrc) + off);
    const float4* v4 = reinterpret_cast<const float4*>(e.V + (size_t)z0 * MPLANE);
    const float sg = (float)e.sigma[0];  // 0 except in the shifted FP32 stage
#pragma unroll 4
    for (int t = threadIdx.x; t < MPL * MPLANE / 4; t += MTHREADS) {
      const int row = t / 12, q = t - row * 12;
      const float4 kv = *reinterpret_cast<const float4*>(rows + row * MROW + 4 * q);
      const float4 xv = __ldg(x4 + t), vv = __ldg(v4 + t);
      out4[t] = make_float4(kv.x + (vv.x - sg) * xv.x, kv.y + (vv.y - sg) * xv.y, kv.z + (vv.z - sg) * xv.z,
                            kv.w + (vv.w - sg) * xv.w);
    }
  } else {
    for (int t = threadIdx.x; t < MPL * MPLANE / 4; t += MTHREADS) {
      const int row = t / 12, q = t - row * 12;
      out4[t] = *reinterpret_cast<const float4*>(rows + row * MROW + 4 * q);
    }
  }
}

}  // namespace

bool mono_grid(const BatchShape& s) {
  return s.uni_nx == MX && s.uni_ny == MY && (s.uni_nz == 40 || s.uni_nz == 48);
}

void mono_xy_fwd(const Batch<float>& b, BRef<float> src, int ncols, int filt, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  mono_fwd_kernel<<<dim3(s.uni_nz / MPL, nc, s.nel), MTHREADS, MSMEM, st>>>(b.d_elems, src, ncols, filt,
                                                                             s.uni_nz);
}

void mono_z(const Batch<float>& b, int mode, int ncols, const double* tkin_override, int filt, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  const dim3 g(MSPEC / ZTHREADS, nc, s.nel);
  if (s.uni_nz == 40) {
    if (mode == ZM_TETER)
      mono_z_kernel<40, ZM_TETER><<<g, ZTHREADS, 0, st>>>(b.d_elems, ncols, tkin_override, filt);
    else if (mode == ZM_MASK)
      mono_z_kernel<40, ZM_MASK><<<g, ZTHREADS, 0, st>>>(b.d_elems, ncols, tkin_override, filt);
    else
      mono_z_kernel<40, ZM_KINETIC><<<g, ZTHREADS, 0, st>>>(b.d_elems, ncols, tkin_override, filt);
  } else {
    if (mode == ZM_TETER)
      mono_z_kernel<48, ZM_TETER><<<g, ZTHREADS, 0, st>>>(b.d_elems, ncols, tkin_override, filt);
    else if (mode == ZM_MASK)
      mono_z_kernel<48, ZM_MASK><<<g, ZTHREADS, 0, st>>>(b.d_elems, ncols, tkin_override, filt);
    else
      mono_z_kernel<48, ZM_KINETIC><<<g, ZTHREADS, 0, st>>>(b.d_elems, ncols, tkin_override, filt);
  }
}

void mono_xy_inv(const Batch<float>& b, int mode, BRef<float> dst, BRef<float> xsrc, int ncols, int filt,
                 cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  const dim3 g(s.uni_nz / MPL, nc, s.nel);
  if (mode == XI_HAMILTONIAN)
    mono_inv_kernel<XI_HAMILTONIAN><<<g, MTHREADS, MSMEM, st>>>(b.d_elems, dst, xsrc, ncols, filt, s.uni_nz);
  else
    mono_inv_kernel<XI_PLAIN><<<g, MTHREADS, MSMEM, st>>>(b.d_elems, dst, xsrc, ncols, filt, s.uni_nz);
}

// Twiddle tables (FP64 on the host, rounded to FP32) and the shared-memory
// opt-in; idempotent.
void init_mono_kernels() {
  static bool done = false;
  if (done) return;
  auto fill = [](float2* w, int n) {
    const double two_pi = 6.283185307179586476925286766559;
    for (int t = 0; t < n; ++t) {
      const double a = two_pi * t / n;
      w[t] = make_float2((float)std::cos(a), (float)-std::sin(a));
    }
  };
  float2 w48[48], w64[64], w40[40];
  fill(w48, 48);
  fill(w64, 64);
  fill(w40, 40);
  if (cudaMemcpyToSymbol(c_w48, w48, sizeof(w48)) != cudaSuccess) return;
  if (cudaMemcpyToSymbol(c_w64, w64, sizeof(w64)) != cudaSuccess) return;
  if (cudaMemcpyToSymbol(c_w40, w40, sizeof(w40)) != cudaSuccess) return;
  cudaFuncSetAttribute((const void*)mono_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MSMEM);
  cudaFuncSetAttribute((const void*)mono_inv_kernel<XI_HAMILTONIAN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)MSMEM);
  cudaFuncSetAttribute((const void*)mono_inv_kernel<XI_PLAIN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       (int)MSMEM);
  done = true;
}

}  // namespace dgdft
