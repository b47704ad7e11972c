// H apply and Teter preconditioner on batches of elements.
//
// Sec. II.B, operation 1: H Psi = -1/2 Lap Psi (FFT) + V_eff Psi (local) +
// sum_p gamma_p b_p <b_p, Psi> (Kleinman-Bylander, Eq. DGvar nonlocal term).
// Sec. II.B, operation 5: the Teter preconditioner, applied per column.
//
// Three passes over HBM per block (a 3-D transform needs one transpose when
// a whole grid does not fit on chip):
//   xy_fwd : per (plane z, vector j): real plane -> r2c along x (as a complex
//            FFT of length nx/2 plus an even/odd split) -> FFT along y;
//   z_mult : per (tile of (y, kx) columns, vector j): FFT along z, multiply by
//            the kinetic symbol |G|^2/2 (or the Teter factor, or the mask of
//            the sphere |G|^2/2 <= ecut for the cutoff's projection), inverse
//            FFT;
//   xy_inv : inverse y, c2r along x, fused epilogue adding V_eff psi and the
//            projector scatter for the points of plane z.
#include <type_traits>

#include "fft.cuh"
#include "dfloat.cuh"
#include "internal.h"

namespace dgdft {

namespace {

template <class real>
__device__ __forceinline__ bool elem_live(const ElemDev<real>& e) {
  return e.state[ST_ACTIVE] != 0;
}
// filt = 1: only elements that precondition with Teter (the others use the
// learned network this iteration)
template <class real>
__device__ __forceinline__ bool elem_live(const ElemDev<real>& e, int filt) {
  return e.state[ST_ACTIVE] != 0 && (filt == 0 || e.state[ST_TETER] != 0);
}

// C[p, j] = v_p^T psi_j for the projectors of the element.
template <class real>
__global__ void proj_coef_kernel(const ElemDev<real>* __restrict__ elems, BRef<real> src, int ncols) {
  const ElemDev<real>& e = elems[blockIdx.z];
  const int p = blockIdx.x;
  if (!elem_live(e) || p >= e.n_proj) return;
  const int nc = ncols > 0 ? ncols : e.m;
  const real* x = resolve(e, src);
  const int beg = e.p_ptr[p], end = e.p_ptr[p + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int j = warp; j < nc; j += nwarp) {
    const real* xj = x + (size_t)j * e.ng;
    real acc = 0;
    for (int q = beg + lane; q < end; q += 32) acc += e.p_val[q] * xj[e.p_idx[q]];
    acc = warp_sum(acc);
    if (lane == 0) e.Ccoef[p + (size_t)j * e.n_proj] = acc;
  }
}

// Pass 1.  real: storage of the vectors; TC: arithmetic; TZ: the stored
// half spectrum.
template <class real, class TC, class TZ, int NH = 0, int NY = 0>
__global__ void xy_fwd_kernel(const ElemDev<real>* __restrict__ elems, BRef<real> src, int ncols, int filt) {
  using C = cplx_t<TC>;
  using R2 = cplx_t<real>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ElemDev<real>& e = elems[blockIdx.z];
  const int z = blockIdx.x, j = blockIdx.y;
  const int nc = ncols > 0 ? ncols : e.m;
  if (!elem_live(e, filt) || z >= e.nz || j >= nc) return;
  const int nh = NH ? NH : e.nh, ny = NY ? NY : e.ny, nxh = nh + 1, row = nxh;
  if (NH && (e.nh != NH || e.ny != NY)) return;  // launched only on uniform batches of this grid
  const unsigned mag_nh = div_magic(nh), mag_nxh = div_magic(nxh);
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + ny * row;
  const R2* plane = reinterpret_cast<const R2*>(resolve(e, src) + (size_t)j * e.ng + (size_t)z * e.nx * ny);
  for (int t = threadIdx.x; t < nh * ny; t += blockDim.x) {
    const int y = (NH ? t / nh : udiv_small(t, mag_nh)), k = t - y * nh;
    const R2 v = plane[t];
    buf0[y * row + k] = cmake<C>((TC)v.x, (TC)v.y);
  }
  __syncthreads();
  const C* tw_h = twp<TC>(e, TW_H);
  const C* tw_x = twp<TC>(e, TW_X);
  int cur = fft_lines_n<C, false, NH>(buf0, buf1, 0, e.px, ny, row, 1, tw_h);
  // even/odd split: X[k] = E[k] + e^{-2 pi i k / nx} O[k], k = 0..nh
  {
    const C* s = cur ? buf1 : buf0;
    C* d = cur ? buf0 : buf1;
    for (int t = threadIdx.x; t < nxh * ny; t += blockDim.x) {
      const int y = (NH ? t / nxh : udiv_small(t, mag_nxh)), k = t - y * nxh;
      const C zk = s[y * row + (k == nh ? 0 : k)];
      const C zc = cconj(s[y * row + (k == 0 ? 0 : nh - k)]);
      const C ev = cscale(cadd(zk, zc), (TC)0.5);
      const C df = csub(zk, zc);
      const C od = cmake<C>((TC)0.5 * df.y, (TC)-0.5 * df.x);  // -i/2 (zk - zc)
      d[y * row + k] = cadd(ev, cmul(tw_x[k], od));
    }
    __syncthreads();
    cur ^= 1;
  }
  cur = fft_lines_n<C, false, NY>(buf0, buf1, cur, e.py, nxh, 1, row, twp<TC>(e, TW_Y));
  const C* res = cur ? buf1 : buf0;
  cplx_t<TZ>* out = reinterpret_cast<cplx_t<TZ>*>(e.Z) + (size_t)j * e.nspec + (size_t)z * nxh * ny;
  for (int t = threadIdx.x; t < nxh * ny; t += blockDim.x) {
    const int y = (NH ? t / nxh : udiv_small(t, mag_nxh)), k = t - y * nxh;
    const C v = res[y * row + k];
    out[t] = cmake<cplx_t<TZ>>((TZ)v.x, (TZ)v.y);
  }
}

constexpr int ZTILE = 32;
constexpr int ZROW = ZTILE + 1;

__device__ __forceinline__ double teter_factor(double s) {
  const double num = 27.0 + s * (18.0 + s * (12.0 + s * 8.0));
  return num / (num + 16.0 * s * s * s * s);
}

// Pass 2, arithmetic and storage in TZ.
template <class real, class TZ, int MODE, int NZ = 0>
__global__ void z_mult_kernel(const ElemDev<real>* __restrict__ elems, int ncols,
                              const double* __restrict__ tkin_override, int filt) {
  using C = cplx_t<TZ>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ElemDev<real>& e = elems[blockIdx.z];
  const int j = blockIdx.y;
  const int nc = ncols > 0 ? ncols : e.m;
  const int nplane = e.nxh * e.ny;
  const unsigned mag_nxh = div_magic(e.nxh);
  const int c0 = blockIdx.x * ZTILE;
  if (!elem_live(e, filt) || j >= nc || c0 >= nplane) return;
  const int nz = NZ ? NZ : e.nz;
  if (NZ && e.nz != NZ) return;  // launched only on uniform batches of this grid
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + nz * ZROW;
  C* zj = reinterpret_cast<C*>(e.Z) + (size_t)j * e.nspec;
  for (int t = threadIdx.x; t < nz * ZTILE; t += blockDim.x) {
    const int z = t / ZTILE, cc = t - z * ZTILE;
    const int c = c0 + cc;
    buf0[z * ZROW + cc] = (c < nplane) ? zj[(size_t)z * nplane + c] : cmake<C>(0, 0);
  }
  __syncthreads();
  const C* tw_z = twp<TZ>(e, TW_Z);
  int cur = fft_lines_n<C, false, NZ>(buf0, buf1, 0, e.pz, ZTILE, 1, ZROW, tw_z);
  {
    C* s = cur ? buf1 : buf0;
    double tk = 1.0;
    if (MODE == ZM_TETER) tk = tkin_override ? tkin_override[j] : e.tkin[j];
    if constexpr (sizeof(TZ) == sizeof(float)) {
      // FP32 symbols and Teter factor: no FP64 arithmetic per point (nor a
      // per-thread FP64 division)
      const float inv_tkf = 1.0f / fmaxf((float)tk, 1e-8f), scalef = (float)e.scale;
      for (int t = threadIdx.x; t < nz * ZTILE; t += blockDim.x) {
        const int gz = t / ZTILE, cc = t - gz * ZTILE;
        const int c = c0 + cc;
        if (c >= nplane) continue;
        const int y = udiv_small(c, mag_nxh), kx = c - y * e.nxh;
        const float g = e.gx2f[kx] + e.gy2f[y] + e.gz2f[gz];
        float f = g;
        if (MODE == ZM_TETER) {
          const float sv = g * inv_tkf;
          const float num = 27.0f + sv * (18.0f + sv * (12.0f + sv * 8.0f));
          f = num / (num + 16.0f * sv * sv * sv * sv);
        } else if (MODE == ZM_MASK) {
          f = (g <= (float)e.ecut) ? 1.0f : 0.0f;
        }
        s[gz * ZROW + cc] = cscale(s[gz * ZROW + cc], (TZ)(f * scalef));
      }
    } else {
      for (int t = threadIdx.x; t < nz * ZTILE; t += blockDim.x) {
        const int gz = t / ZTILE, cc = t - gz * ZTILE;
        const int c = c0 + cc;
        if (c >= nplane) continue;
        const int y = udiv_small(c, mag_nxh), kx = c - y * e.nxh;
        const double g = e.gx2[kx] + e.gy2[y] + e.gz2[gz];
        double f = (MODE == ZM_KINETIC) ? g
                   : (MODE == ZM_TETER) ? teter_factor(g / fmax(tk, 1e-8))
                                        : ((g <= e.ecut) ? 1.0 : 0.0);
        f *= e.scale;
        s[gz * ZROW + cc] = cscale(s[gz * ZROW + cc], (TZ)f);
      }
    }
    __syncthreads();
  }
  cur = fft_lines_n<C, true, NZ>(buf0, buf1, cur, e.pz, ZTILE, 1, ZROW, tw_z);
  const C* res = cur ? buf1 : buf0;
  for (int t = threadIdx.x; t < nz * ZTILE; t += blockDim.x) {
    const int z = t / ZTILE, cc = t - z * ZTILE;
    const int c = c0 + cc;
    if (c < nplane) zj[(size_t)z * nplane + c] = res[z * ZROW + cc];
  }
}

// Pass 3: Z (TZ) -> arithmetic TC -> vectors (real), with the epilogue.
template <class real, class TZ, class TC, int MODE, int NH = 0, int NY = 0>
__global__ void xy_inv_kernel(const ElemDev<real>* __restrict__ elems, BRef<real> dst,
                              BRef<real> xsrc, int ncols, int filt) {
  using C = cplx_t<TC>;
  using R2 = cplx_t<real>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const ElemDev<real>& e = elems[blockIdx.z];
  const int z = blockIdx.x, j = blockIdx.y;
  const int nc = ncols > 0 ? ncols : e.m;
  if (!elem_live(e, filt) || z >= e.nz || j >= nc) return;
  const int nh = NH ? NH : e.nh, ny = NY ? NY : e.ny, nxh = nh + 1, row = nxh;
  if (NH && (e.nh != NH || e.ny != NY)) return;  // launched only on uniform batches of this grid
  const unsigned mag_nh = div_magic(nh), mag_nxh = div_magic(nxh);
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + ny * row;
  const cplx_t<TZ>* in = reinterpret_cast<const cplx_t<TZ>*>(e.Z) + (size_t)j * e.nspec + (size_t)z * nxh * ny;
  for (int t = threadIdx.x; t < nxh * ny; t += blockDim.x) {
    const int y = (NH ? t / nxh : udiv_small(t, mag_nxh)), k = t - y * nxh;
    const cplx_t<TZ> v = in[t];
    buf0[y * row + k] = cmake<C>((TC)v.x, (TC)v.y);
  }
  __syncthreads();
  const C* tw_x = twp<TC>(e, TW_X);
  int cur = fft_lines_n<C, true, NY>(buf0, buf1, 0, e.py, nxh, 1, row, twp<TC>(e, TW_Y));
  // recombine the half spectrum into E + i O for the length-nh inverse
  {
    const C* s = cur ? buf1 : buf0;
    C* d = cur ? buf0 : buf1;
    for (int t = threadIdx.x; t < nh * ny; t += blockDim.x) {
      const int y = (NH ? t / nh : udiv_small(t, mag_nh)), k = t - y * nh;
      const C xk = s[y * row + k];
      const C xc = cconj(s[y * row + nh - k]);
      const C ev = cscale(cadd(xk, xc), (TC)0.5);
      const C od = cmul(cscale(csub(xk, xc), (TC)0.5), cconj(tw_x[k]));
      d[y * row + k] = cmake<C>(ev.x - od.y, ev.y + od.x);
    }
    __syncthreads();
    cur ^= 1;
  }
  cur = fft_lines_n<C, true, NH>(buf0, buf1, cur, e.px, ny, row, 1, twp<TC>(e, TW_H));
  C* res = cur ? buf1 : buf0;
  const size_t plane_off = (size_t)j * e.ng + (size_t)z * e.nx * ny;
  if (MODE == XI_HAMILTONIAN) {
    // Kleinman-Bylander scatter for the support points of this plane
    if (e.n_sup > 0) {
      const int sb = e.s_plane[z], se = e.s_plane[z + 1];
      const real* cj = e.Ccoef + (size_t)j * e.n_proj;
      TC* rres = reinterpret_cast<TC*>(res);
      for (int s = sb + threadIdx.x; s < se; s += blockDim.x) {
        TC acc = 0;
        for (int q = e.s_ptr[s]; q < e.s_ptr[s + 1]; ++q) acc += (TC)e.s_gv[q] * (TC)cj[e.s_proj[q]];
        const int off = e.s_off[s];
        const int nx = 2 * nh;
        const int y = off / nx, x = off - y * nx;
        rres[2 * (y * row) + x] += acc;
      }
      __syncthreads();
    }
    const R2* xp = reinterpret_cast<const R2*>(resolve(e, xsrc) + plane_off);
    const R2* vp = reinterpret_cast<const R2*>(e.V + (size_t)z * e.nx * ny);
    R2* op = reinterpret_cast<R2*>(resolve(e, dst) + plane_off);
    const TC sg = (TC)e.sigma[0];  // 0 except in the shifted FP32 stage
    for (int t = threadIdx.x; t < nh * ny; t += blockDim.x) {
      const int y = (NH ? t / nh : udiv_small(t, mag_nh)), k = t - y * nh;
      const C kv = res[y * row + k];
      const R2 xv = xp[t];
      const R2 vv = vp[t];
      op[t] = cmake<R2>((real)(kv.x + ((TC)vv.x - sg) * (TC)xv.x), (real)(kv.y + ((TC)vv.y - sg) * (TC)xv.y));
    }
  } else {
    R2* op = reinterpret_cast<R2*>(resolve(e, dst) + plane_off);
    for (int t = threadIdx.x; t < nh * ny; t += blockDim.x) {
      const int y = (NH ? t / nh : udiv_small(t, mag_nh)), k = t - y * nh;
      const C v = res[y * row + k];
      op[t] = cmake<R2>((real)v.x, (real)v.y);
    }
  }
}

template <class T> size_t plane_smem(const BatchShape& s) {
  return 2 * sizeof(cplx_t<T>) * (size_t)s.max_ny * s.max_nxh;
}
template <class T> size_t zcol_smem(const BatchShape& s) {
  return 2 * sizeof(cplx_t<T>) * (size_t)s.max_nz * ZROW;
}

// Pass launchers: on a batch whose elements share one grid of a supported
// shape (the monolayer extended elements, 48 x 64 x 40 and 48 x 64 x 48) the
// register-resident FP32 kernels of fft_mono.cu, or (FP64 arithmetic) these
// kernels specialised for those line lengths at compile time; otherwise the
// kernels that follow each element's runtime plan.
template <class real, class TC, class TZ>
void launch_xy_fwd(const Batch<real>& b, BRef<real> src, int ncols, int filt, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  const dim3 g(s.max_nz, nc, s.nel);
  if constexpr (std::is_same_v<real, float> && std::is_same_v<TC, float> && std::is_same_v<TZ, float>) {
    if (mono_grid(s)) return mono_xy_fwd(b, src, ncols, filt, st);
  }
  const size_t sm = plane_smem<TC>(s);
  if (s.uni_nx == 48 && s.uni_ny == 64)
    xy_fwd_kernel<real, TC, TZ, 24, 64><<<g, 256, sm, st>>>(b.d_elems, src, ncols, filt);
  else
    xy_fwd_kernel<real, TC, TZ><<<g, 256, sm, st>>>(b.d_elems, src, ncols, filt);
}

template <class real, class TZ, int MODE>
void launch_z_mult(const Batch<real>& b, int ncols, const double* tkin_override, int filt, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  if constexpr (std::is_same_v<real, float> && std::is_same_v<TZ, float>) {
    if (mono_grid(s)) return mono_z(b, MODE, ncols, tkin_override, filt, st);
  }
  const dim3 g((s.max_nplane + ZTILE - 1) / ZTILE, nc, s.nel);
  const size_t sm = zcol_smem<TZ>(s);
  if (s.uni_nz == 40)
    z_mult_kernel<real, TZ, MODE, 40><<<g, 256, sm, st>>>(b.d_elems, ncols, tkin_override, filt);
  else if (s.uni_nz == 48)
    z_mult_kernel<real, TZ, MODE, 48><<<g, 256, sm, st>>>(b.d_elems, ncols, tkin_override, filt);
  else
    z_mult_kernel<real, TZ, MODE><<<g, 256, sm, st>>>(b.d_elems, ncols, tkin_override, filt);
}

template <class real, class TZ, class TC, int MODE>
void launch_xy_inv(const Batch<real>& b, BRef<real> dst, BRef<real> src, int ncols, int filt, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  const dim3 g(s.max_nz, nc, s.nel);
  if constexpr (std::is_same_v<real, float> && std::is_same_v<TZ, float> && std::is_same_v<TC, float>) {
    if (mono_grid(s)) return mono_xy_inv(b, MODE, dst, src, ncols, filt, st);
  }
  const size_t sm = plane_smem<TC>(s);
  if (s.uni_nx == 48 && s.uni_ny == 64)
    xy_inv_kernel<real, TZ, TC, MODE, 24, 64><<<g, 256, sm, st>>>(b.d_elems, dst, src, ncols, filt);
  else
    xy_inv_kernel<real, TZ, TC, MODE><<<g, 256, sm, st>>>(b.d_elems, dst, src, ncols, filt);
}

}  // namespace

template <class real, class F>
void apply_h_prec(const Batch<real>& b, BRef<real> src, BRef<real> dst, int ncols, cudaStream_t st) {
  const BatchShape& s = b.s;
  const int nc = ncols > 0 ? ncols : s.max_m;
  if (s.max_nproj > 0)
    proj_coef_kernel<real><<<dim3(s.max_nproj, 1, s.nel), 128, 0, st>>>(b.d_elems, src, ncols);
  (void)nc;
  launch_xy_fwd<real, F, F>(b, src, ncols, 0, st);
  launch_z_mult<real, F, ZM_KINETIC>(b, ncols, nullptr, 0, st);
  launch_xy_inv<real, F, real, XI_HAMILTONIAN>(b, dst, src, ncols, 0, st);
}

// FP64 vectors with the transforms in double-float arithmetic (FP32 pairs,
// ~2^-46 relative per operation): the FP64 waves of the mixed form, whose
// FP64 FFT passes would run on the FP64 pipe (1/55 of the FP32 rate here).
void apply_h_dfloat(const Batch<double>& b, BRef<double> src, BRef<double> dst, int ncols, cudaStream_t st) {
  const BatchShape& s = b.s;
  if (s.max_nproj > 0)
    proj_coef_kernel<double><<<dim3(s.max_nproj, 1, s.nel), 128, 0, st>>>(b.d_elems, src, ncols);
  launch_xy_fwd<double, dff, dff>(b, src, ncols, 0, st);
  launch_z_mult<double, dff, ZM_KINETIC>(b, ncols, nullptr, 0, st);
  launch_xy_inv<double, dff, dff, XI_HAMILTONIAN>(b, dst, src, ncols, 0, st);
}

// fwd64: run the forward transform (passes 1-2) in FP64 with an FP64
// intermediate even for FP32 vectors (the rounding of the forward transform
// is what |G|^2/2 amplifies); pass 3 stays in the working precision.
template <class real>
void launch_apply_h(const Batch<real>& b, BRef<real> src, BRef<real> dst, int ncols, cudaStream_t st,
                    bool fwd64) {
  if constexpr (std::is_same<real, double>::value) {
    if (b.s.dfloat) {
      apply_h_dfloat(b, src, dst, ncols, st);
      return;
    }
  }
  if (fwd64)
    apply_h_prec<real, double>(b, src, dst, ncols, st);
  else
    apply_h_prec<real, real>(b, src, dst, ncols, st);
}

// The preconditioner's accuracy does not limit convergence: all passes run
// in the working precision.
template <class real>
void launch_teter(const Batch<real>& b, BRef<real> src, BRef<real> dst, const double* tkin_override,
                  int ncols, cudaStream_t st, int only_teter_elems) {
  const int f = only_teter_elems;
  if constexpr (std::is_same<real, double>::value) {
    if (b.s.dfloat) {
      launch_xy_fwd<double, dff, dff>(b, src, ncols, f, st);
      launch_z_mult<double, dff, ZM_TETER>(b, ncols, tkin_override, f, st);
      launch_xy_inv<double, dff, dff, XI_PLAIN>(b, dst, src, ncols, f, st);
      return;
    }
  }
  launch_xy_fwd<real, real, real>(b, src, ncols, f, st);
  launch_z_mult<real, real, ZM_TETER>(b, ncols, tkin_override, f, st);
  launch_xy_inv<real, real, real, XI_PLAIN>(b, dst, src, ncols, f, st);
}

// Sphere-cutoff projection: the grid passes of the Teter preconditioner
// with the mask |G|^2/2 <= ecut as the multiplier.  FP64 vectors: FP64
// passes, or double-float passes in the mixed form's FP64 waves; the mask is
// decided on the FP64 symbols of the kinetic term, in the same order.
void launch_project(const Batch<double>& b, BRef<double> src, BRef<double> dst, int ncols, cudaStream_t st) {
  if (b.s.dfloat) {
    launch_xy_fwd<double, dff, dff>(b, src, ncols, 0, st);
    launch_z_mult<double, dff, ZM_MASK>(b, ncols, nullptr, 0, st);
    launch_xy_inv<double, dff, dff, XI_PLAIN>(b, dst, src, ncols, 0, st);
    return;
  }
  launch_xy_fwd<double, double, double>(b, src, ncols, 0, st);
  launch_z_mult<double, double, ZM_MASK>(b, ncols, nullptr, 0, st);
  launch_xy_inv<double, double, double, XI_PLAIN>(b, dst, src, ncols, 0, st);
}
// FP32 vectors (the mixed form's FP32 stage): FP32 passes (the register-
// resident ones on the monolayer grids), the mask decided on the FP32
// symbols; a frequency within FP32 rounding of the sphere may be decided
// differently from the FP64 stage, whose projections decide the result.
void launch_project(const Batch<float>& b, BRef<float> src, BRef<float> dst, int ncols, cudaStream_t st) {
  launch_xy_fwd<float, float, float>(b, src, ncols, 0, st);
  launch_z_mult<float, float, ZM_MASK>(b, ncols, nullptr, 0, st);
  launch_xy_inv<float, float, float, XI_PLAIN>(b, dst, src, ncols, 0, st);
}

// Allow the plane and column kernels the full opt-in shared memory once.
template <class real> static void opt_in_smem_t() {
  opt_in_dynamic_smem((const void*)xy_fwd_kernel<real, double, double, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_fwd_kernel<real, real, real, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<real, double, real, XI_HAMILTONIAN, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<real, real, real, XI_HAMILTONIAN, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<real, real, real, XI_PLAIN, 24, 64>);
  for (int k = 0; k < 2; ++k) {
    opt_in_dynamic_smem(k ? (const void*)z_mult_kernel<real, double, ZM_KINETIC, 48>
                          : (const void*)z_mult_kernel<real, double, ZM_KINETIC, 40>);
    opt_in_dynamic_smem(k ? (const void*)z_mult_kernel<real, real, ZM_KINETIC, 48>
                          : (const void*)z_mult_kernel<real, real, ZM_KINETIC, 40>);
    opt_in_dynamic_smem(k ? (const void*)z_mult_kernel<real, real, ZM_TETER, 48>
                          : (const void*)z_mult_kernel<real, real, ZM_TETER, 40>);
  }
  opt_in_dynamic_smem((const void*)xy_fwd_kernel<real, double, double>);
  opt_in_dynamic_smem((const void*)xy_fwd_kernel<real, real, real>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<real, double, real, XI_HAMILTONIAN>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<real, real, real, XI_HAMILTONIAN>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<real, real, real, XI_PLAIN>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<real, double, ZM_KINETIC>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<real, real, ZM_KINETIC>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<real, real, ZM_TETER>);
}
// Raise a kernel's dynamic shared-memory limit to the device's opt-in
// maximum minus the kernel's static shared memory.
void opt_in_dynamic_smem(const void* kernel) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kernel) != cudaSuccess) return;
  cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
}

static void opt_in_smem_dfloat() {
  opt_in_dynamic_smem((const void*)xy_fwd_kernel<double, dff, dff, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_fwd_kernel<double, dff, dff>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<double, dff, dff, XI_HAMILTONIAN, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<double, dff, dff, XI_HAMILTONIAN>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<double, dff, dff, XI_PLAIN, 24, 64>);
  opt_in_dynamic_smem((const void*)xy_inv_kernel<double, dff, dff, XI_PLAIN>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_KINETIC, 40>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_KINETIC, 48>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_KINETIC>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_TETER, 40>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_TETER, 48>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_TETER>);
}

void init_hamiltonian_kernels() {
  init_mono_kernels();
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, double, ZM_MASK, 40>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, double, ZM_MASK, 48>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, double, ZM_MASK>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_MASK, 40>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_MASK, 48>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<double, dff, ZM_MASK>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<float, float, ZM_MASK, 40>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<float, float, ZM_MASK, 48>);
  opt_in_dynamic_smem((const void*)z_mult_kernel<float, float, ZM_MASK>);
  opt_in_smem_t<double>();
  opt_in_smem_t<float>();
  opt_in_smem_dfloat();
}

// One pass of the H apply in isolation (0: xy forward, 1: z multiply,
// 2: xy inverse with epilogue), for stage timing.
template <class real>
void launch_h_pass(const Batch<real>& b, int pass, BRef<real> src, BRef<real> dst, int ncols, cudaStream_t st) {
  using F = real;
  using I = real;
  if (pass == 0)
    launch_xy_fwd<real, F, F>(b, src, ncols, 0, st);
  else if (pass == 1)
    launch_z_mult<real, F, ZM_KINETIC>(b, ncols, nullptr, 0, st);
  else
    launch_xy_inv<real, F, I, XI_HAMILTONIAN>(b, dst, src, ncols, 0, st);
}
template void launch_h_pass<double>(const Batch<double>&, int, BRef<double>, BRef<double>, int, cudaStream_t);
template void launch_h_pass<float>(const Batch<float>&, int, BRef<float>, BRef<float>, int, cudaStream_t);

template <class real>
void launch_proj_coef(const Batch<real>& b, BRef<real> src, int ncols, cudaStream_t st) {
  if (b.s.max_nproj > 0)
    proj_coef_kernel<real><<<dim3(b.s.max_nproj, 1, b.s.nel), 128, 0, st>>>(b.d_elems, src, ncols);
}
template void launch_proj_coef<double>(const Batch<double>&, BRef<double>, int, cudaStream_t);
template void launch_proj_coef<float>(const Batch<float>&, BRef<float>, int, cudaStream_t);

template void launch_apply_h<double>(const Batch<double>&, BRef<double>, BRef<double>, int, cudaStream_t, bool);
template void launch_apply_h<float>(const Batch<float>&, BRef<float>, BRef<float>, int, cudaStream_t, bool);
template void launch_teter<double>(const Batch<double>&, BRef<double>, BRef<double>, const double*, int,
                                   cudaStream_t, int);
template void launch_teter<float>(const Batch<float>&, BRef<float>, BRef<float>, const double*, int,
                                  cudaStream_t, int);

}  // namespace dgdft
