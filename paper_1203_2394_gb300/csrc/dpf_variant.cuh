// Launchers of one compiled (precision, d1, d2, dy) variant of the step.
#pragma once

#include <cmath>
#include <cstring>

#include "dpf_pf.cuh"
#include "dpf_std.cuh"
#include "dpf_step_warp.cuh"
#include "dpf_outer.cuh"

namespace dpf {

inline int threads_for(int M) { return ((M + 31) / 32) * 32; }

// The outer stage of a step (the outer reduction and the global resampling, in one
// cooperative launch: fused_outer_kernel), for every filter kind. `arrive` is the
// grid barrier's counter (null for the two-launch batched form).
template <typename T>
void fill_outer_args(Ctx& x, double* mean_out, double* logz_out, unsigned int* arrive, void* out) {
    FusedOuterArgs<T>& a = *(FusedOuterArgs<T>*)out;
    a = FusedOuterArgs<T>{};
    OuterArgs<T>& o = a.o;
    o.lw = (const T*)x.lw;
    o.xm = (const T*)x.xm;
    o.zm = (const T*)x.zm;
    o.N = x.N;
    o.d1 = x.d1;
    o.d2 = x.d2;
    o.lwmax_key = x.lwmax_key;
    o.lwmax_t = (T*)x.lwmax_t;
    o.Csum = x.Csum;
    o.done = x.done;
    o.partials = x.partials;
    o.stats = x.stats;
    o.perm = (const int*)(x.stats + 4 + x.d);  // the permutation lives after the statistics
    o.mean_out = mean_out;
    o.logz_out = logz_out;
    o.err = x.err;
    a.w_out = (T*)x.wout;
    a.anc = x.anc;
    a.ctot = x.ctot;
    a.arrive = arrive;
    a.shift = 62 - ceil_log2_i(x.N);
    a.logN = std::log((double)x.N);
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    a.t = (uint32_t)(x.t + 1);
    a.withhold = -1;
    a.host_stats = x.host_out ? x.hstats_dev : nullptr;
  }

template <typename T, int D1, int D2>
dpf_status outer_stage(Ctx& x, double* mean_out, double* logz_out, cudaStream_t st) {
    FusedOuterArgs<T> a;
    fill_outer_args<T>(x, mean_out, logz_out, x.done + 1, &a);
    a.nwork = fused_outer_grid<T, D1, D2>(x.N);
    return cuda_error(fused_outer_launch<T, D1, D2>(a, st), "outer stage launch");
  }

// XZM: 0 = kernels for both x-transition kinds, 1 = only the general (x depends on z) kernels.
template <typename T, int D1, int D2, int DY, int XZM = 0>
struct VariantImpl {
  typedef MC<T, D1, D2, DY> Const;

  static dpf_status make_const(const HostModel& h, std::vector<unsigned char>& out) {
    Const c;
    memset(&c, 0, sizeof(c));
    auto cp = [](const std::vector<double>& src, T* dst, int n) {
      for (int q = 0; q < n; ++q) dst[q] = (T)src[q];
    };
    cp(h.Axx, &c.Axx[0][0], D1 * D1);
    cp(h.Azx, &c.Azx[0][0], D2 * D1);
    cp(h.Azz, &c.Azz[0][0], D2 * D2);
    cp(h.Lqx, &c.Lqx[0][0], D1 * D1);
    cp(h.LqxInv, &c.LqxInv[0][0], D1 * D1);
    cp(h.Lqz, &c.Lqz[0][0], D2 * D2);
    cp(h.WAxz, &c.WAxz[0][0], D1 * D2);
    cp(h.Hx, &c.Hx[0][0], DY * D1);
    cp(h.Hz, &c.Hz[0][0], DY * D2);
    cp(h.LrInv, &c.LrInv[0][0], DY * DY);
    cp(h.LrHz, &c.LrHz[0][0], DY * D2);
    cp(h.HzAzz, &c.HzAzz[0][0], DY * D2);
    cp(h.HzAzx, &c.HzAzx[0][0], DY * D1);
    cp(h.Ls, &c.Ls[0][0], DY * DY);
    cp(h.K, &c.K[0][0], D2 * DY);
    cp(h.m0x, c.m0x, D1);
    cp(h.m0z, c.m0z, D2);
    cp(h.Lp0x, &c.Lp0x[0][0], D1 * D1);
    cp(h.G0, &c.G0[0][0], D2 * D1);
    cp(h.Lp0c, &c.Lp0c[0][0], D2 * D2);
    c.ga = (T)h.ga;
    c.gb = (T)h.gb;
    c.qc = (T)h.qc;
    c.lognorm_y = (T)h.lognorm_y;
    c.growth = h.growth;
    c.quad = h.quad;
    c.diag_qz = 1;
    for (int r = 0; r < D2; ++r)
      for (int q = 0; q < r; ++q) c.diag_qz &= (h.Lqz[r * D2 + q] == 0.0);
    out.resize(sizeof(c));
    memcpy(out.data(), &c, sizeof(c));
    return DPF_OK;
  }

  static const Const& cst(const Ctx& x) { return *reinterpret_cast<const Const*>(x.mconst.data()); }

  // The warp-per-group kernel serves M <= 256 when every staged row is a
  // multiple of 16 bytes (bulk copies); the block kernel serves the rest.
  static bool warp_path(int M, int L) {
    const size_t s = sizeof(T);
    const int ppl = M <= 32 ? 1 : M <= 64 ? 2 : M <= 128 ? 4 : 8;
    return M <= 256 && M % ppl == 0 && (M * s) % 16 == 0 && (L * s) % 16 == 0 &&
           (L * D1 * s) % 16 == 0;
  }
  static size_t smem(int M, int L, bool xz, int nt) {
    if (XZM == 1) xz = true;
    if (warp_path(M, L))
      return xz ? warp_geometry<T, D1, D2, DY, true>(M, L, nullptr)
                : warp_geometry<T, D1, D2, DY, false>(M, L, nullptr);
    return xz ? step_geometry<T, D1, D2, DY, true>(M, L, nt, nullptr)
              : step_geometry<T, D1, D2, DY, false>(M, L, nt, nullptr);
  }
  static int xpad() { return (int)((D1 * sizeof(T) + 15) / 16 * 16 / sizeof(T)); }

  static dpf_status init(Ctx& x) {
    const Key key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    init_kernel<T, D1, D2, DY><<<(unsigned)x.N, threads_for(x.M), 0, x.stream>>>(
        cst(x), (T*)x.z[0], (T*)x.lq[0], (T*)x.x[0], x.N, x.M, x.xp, key);
    return cuda_error(cudaGetLastError(), "init kernel launch");
  }

  template <bool XZ, int PPT, int MAXNT, bool BULK>
  static dpf_status launch_step(Ctx& x, StepArgs<T>& a) {
    auto k = step_kernel<T, D1, D2, DY, XZ, PPT, MAXNT, BULK>;
    static bool attr_done = false;
    if (!attr_done) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
      attr_done = true;
    }
    const int nt = threads_for((x.M + PPT - 1) / PPT);
    const size_t sm = step_geometry<T, D1, D2, DY, XZ>(x.M, x.L, nt, &a, a.first != 0);
    if (x.grid_step == 0) {  // persistent grid: as many CTAs as fit on the device at once
      int nb = 0, dev = 0, nsm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nt, sm);
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return cuda_error(e, "step kernel occupancy");
      x.grid_step = (nb > 0 ? nb : 1) * nsm;
    }
    const long long grid = std::min<long long>(x.N, x.grid_step);
    k<<<(unsigned)grid, nt, sm, x.stream>>>(cst(x), a);
    return cuda_error(cudaGetLastError(), "step kernel launch");
  }

  template <bool XZ, int PPL, int MF>
  static dpf_status launch_warp_mf(Ctx& x, StepArgs<T>& a, cudaStream_t stream = nullptr) {
    auto k = step_warp_kernel<T, D1, D2, DY, XZ, PPL, MF>;
    static bool attr_done = false;
    if (!attr_done) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
      attr_done = true;
    }
    const size_t sm = warp_geometry<T, D1, D2, DY, XZ>(x.M, x.L, &a, a.first != 0);
    if (x.grid_step == 0 || x.grid_kernel != (const void*)k) {
      // persistent grid: as many CTAs of this kernel as fit on the device at once
      int nb = 0, dev = 0, nsm = 0;
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, WARPS_PER_CTA * 32, sm);
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return cuda_error(e, "step kernel occupancy");
      x.grid_step = (nb > 0 ? nb : 1) * nsm;
      x.grid_kernel = (const void*)k;
    }
    const long long grid = std::min<long long>((x.N + WARPS_PER_CTA - 1) / WARPS_PER_CTA, x.grid_step);
    k<<<(unsigned)grid, WARPS_PER_CTA * 32, sm, stream ? stream : x.stream>>>(cst(x), a);
    return cuda_error(cudaGetLastError(), "step kernel launch");
  }
  // M = 32 PPL (every lane full) takes the kernel compiled for that M
  template <bool XZ, int PPL>
  static dpf_status launch_warp(Ctx& x, StepArgs<T>& a) {
    if (x.M == 32 * PPL) return launch_warp_mf<XZ, PPL, 32 * PPL>(x, a);
    return launch_warp_mf<XZ, PPL, 0>(x, a);
  }

  template <bool XZ>
  static dpf_status launch_xz(Ctx& x, StepArgs<T>& a) {
    if (!warp_path(x.M, x.L)) return launch_step<XZ, 1, 1024, false>(x, a);
    if (x.M <= 32) return launch_warp<XZ, 1>(x, a);
    if (x.M <= 64) return launch_warp<XZ, 2>(x, a);
    if (x.M <= 128) return launch_warp<XZ, 4>(x, a);
    return launch_warp<XZ, 8>(x, a);
  }

  static void fill_args(Ctx& x, StepArgs<T>& a) {
    const long long t = x.t + 1;  // the step being taken
    const int so = (int)((t + 2) % 2), sn = (int)((t + 1) % 2);  // slots of t-2 and t-1
    // first step, or the inner update already done (learned proposal): the look-ahead
    // starts from the materialised state of t-1 in slot sn (slot 0 at t = 1)
    const bool first = (t == 1) || x.la_only;
    a.la_only = (t > 1 && x.la_only) ? 1 : 0;
    a.z_old = (const T*)x.z[first ? sn : so];
    a.lq_old = (const T*)x.lq[first ? sn : so];
    a.x_old = (const T*)x.x[first ? sn : so];
    a.z_new = (T*)x.z[sn];
    a.lq_new = (T*)x.lq[sn];
    a.x_new = (T*)x.x[sn];
    a.lwh_old = (const T*)x.lwh[(t + 1) % 2];
    a.xbb_old = (const T*)x.xbb[(t + 1) % 2];
    a.lwh_new = (T*)x.lwh[t % 2];
    a.xbb_new = (T*)x.xbb[t % 2];
    a.anc = x.anc;
    a.sel = x.sel;
    a.lw = (T*)x.lw;
    a.xm = (T*)x.xm;
    a.zm = (T*)x.zm;
    a.y_prev = (const T*)x.yb + ((t + 1) % 2) * x.dy;
    a.y_cur = (const T*)x.yb + (t % 2) * x.dy;
    a.lwmax_key = x.lwmax_key;
    a.Csum = x.Csum;
    a.dbg_b = x.debug ? x.dbg_b : nullptr;
    a.err = x.err;
    a.N = x.N;
    a.M = x.M;
    a.L = x.L;
    a.t = (uint32_t)t;
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    const HostModel& h = x.hm;
    a.gcos_prev = h.growth ? (T)(h.gc * std::cos(h.gw * (double)(t - 2))) : T(0);
    a.gcos_cur = h.growth ? (T)(h.gc * std::cos(h.gw * (double)(t - 1))) : T(0);
    a.first = first ? 1 : 0;
    a.scaleM = (T)std::ldexp(1.0, 31 - ceil_log2_i(x.M));
    a.scaleL = (T)std::ldexp(1.0, 31 - ceil_log2_i(x.L));
    a.logM = (T)std::log((double)x.M);
    a.logL = (T)std::log((double)x.L);
    a.glist = x.glist_cur;
    a.gcount = x.gcount_cur;
    a.gskip = x.gskip_cur;
  }

  static bool use_xz(const Ctx& x) { return XZM == 1 || x.hm.xz; }

  static dpf_status step(Ctx& x, int) {
    StepArgs<T> a{};
    fill_args(x, a);
    if constexpr (XZM == 1) return launch_xz<true>(x, a);
    else return use_xz(x) ? launch_xz<true>(x, a) : launch_xz<false>(x, a);
  }

  // ---- many filters of this variant in one launch per PPL class ----
  static int ppl_for(int M) { return M <= 32 ? 1 : M <= 64 ? 2 : M <= 128 ? 4 : 8; }

  // A batched member's step as its own launch of the single-filter kernel on stream s,
  // from its batched launch arguments, at `ppl` inner particles per lane.
  template <bool XZ>
  static dpf_status single_xz(Ctx& x, StepArgs<T>& a, int ppl, cudaStream_t s) {
    switch (ppl) {
      case 1: return x.M == 32 ? launch_warp_mf<XZ, 1, 32>(x, a, s) : launch_warp_mf<XZ, 1, 0>(x, a, s);
      case 2: return x.M == 64 ? launch_warp_mf<XZ, 2, 64>(x, a, s) : launch_warp_mf<XZ, 2, 0>(x, a, s);
      case 4: return x.M == 128 ? launch_warp_mf<XZ, 4, 128>(x, a, s) : launch_warp_mf<XZ, 4, 0>(x, a, s);
      default: return x.M == 256 ? launch_warp_mf<XZ, 8, 256>(x, a, s) : launch_warp_mf<XZ, 8, 0>(x, a, s);
    }
  }
  static dpf_status single_launch(Ctx& x, const void* args, int ppl, bool xz, cudaStream_t s) {
    StepArgs<T> a;
    memcpy(&a, args, sizeof(a));
    if constexpr (XZM == 1) return single_xz<true>(x, a, ppl, s);
    else return xz ? single_xz<true>(x, a, ppl, s) : single_xz<false>(x, a, ppl, s);
  }

  // Per-filter launch arguments for a batched step (y rows given by the batch).
  static void batch_args(Ctx& x, const void* y_prev, const void* y_cur, bool xz, void* out) {
    StepArgs<T> a{};
    fill_args(x, a);
    a.y_prev = (const T*)y_prev;
    a.y_cur = (const T*)y_cur;
    if (xz)
      warp_geometry<T, D1, D2, DY, true>(x.M, x.L, &a, a.first != 0);
    else
      warp_geometry<T, D1, D2, DY, false>(x.M, x.L, &a, a.first != 0);
    memcpy(out, &a, sizeof(a));
  }
  static size_t region_bytes(int M, int L, bool xz) {
    return (xz ? warp_geometry<T, D1, D2, DY, true>(M, L, nullptr)
               : warp_geometry<T, D1, D2, DY, false>(M, L, nullptr)) / WARPS_PER_CTA;
  }

  template <bool XZ, int PPL, bool SHARED, int MF>
  static dpf_status batch_kernel(const BatchLaunch& b, cudaStream_t s, int* occ) {
    auto k = step_warp_batch_kernel<T, D1, D2, DY, XZ, PPL, SHARED, MF>;
    static bool attr_done = false;
    if (!attr_done) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
      attr_done = true;
    }
    if (occ) {
      cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, WARPS_PER_CTA * 32, b.smem);
      return cuda_error(e, "batch kernel occupancy");
    }
    Const mc1;
    if (SHARED) memcpy(&mc1, b.mc_shared, sizeof(Const));
    else memset(&mc1, 0, sizeof(Const));
    k<<<b.grid, WARPS_PER_CTA * 32, b.smem, s>>>(mc1, (const Const*)b.mcs, (const StepArgs<T>*)b.descs,
                                                b.fstart, b.F, b.chunk, b.region);
    return cuda_error(cudaGetLastError(), "batch step kernel launch");
  }
  template <bool XZ, int PPL, bool SHARED>
  static dpf_status batch_mf(const BatchLaunch& b, cudaStream_t s, int* occ) {
    return b.mf ? batch_kernel<XZ, PPL, SHARED, 32 * PPL>(b, s, occ) : batch_kernel<XZ, PPL, SHARED, 0>(b, s, occ);
  }
  template <bool XZ, bool SHARED>
  static dpf_status batch_ppl2(const BatchLaunch& b, cudaStream_t s, int* occ) {
    switch (b.ppl) {
      case 1: return batch_mf<XZ, 1, SHARED>(b, s, occ);
      case 2: return batch_mf<XZ, 2, SHARED>(b, s, occ);
      case 4: return batch_mf<XZ, 4, SHARED>(b, s, occ);
      default: return batch_mf<XZ, 8, SHARED>(b, s, occ);
    }
  }
  template <bool XZ>
  static dpf_status batch_ppl(const BatchLaunch& b, cudaStream_t s, int* occ) {
    return b.mc_shared ? batch_ppl2<XZ, true>(b, s, occ) : batch_ppl2<XZ, false>(b, s, occ);
  }
  // Launch (occ == nullptr) or query the blocks per SM (occ != nullptr).
  static dpf_status batch_launch(const BatchLaunch& b, cudaStream_t s, int* occ) {
    if constexpr (XZM == 1) return batch_ppl<true>(b, s, occ);
    else return b.xz ? batch_ppl<true>(b, s, occ) : batch_ppl<false>(b, s, occ);
  }

  // Arguments of the outer stage that follows the coming step (both of its
  // batched launches read them).
  static void outer_args(Ctx& x, double* mean_out, double* logz_out, void* out) {
    fill_outer_args<T>(x, mean_out, logz_out, nullptr, out);
  }

  // CTAs of the filter's outer stage (the same in the single and batched forms).
  static int outer_ctas(long long N) { return fused_outer_grid<T, D1, D2>(N); }

  static dpf_status outer(Ctx& x, double* mean_out, double* logz_out, cudaStream_t st) {
    return outer_stage<T, D1, D2>(x, mean_out, logz_out, st);
  }

  // The outer sums of F filters of this variant in one launch (device arguments,
  // cstart[F] CTAs in all).
  static dpf_status outer_batch(const void* args, const int* cstart, int nctas, int F, cudaStream_t st) {
    outer_sums_batch_kernel<T, D1, D2><<<nctas, OF_NT, 0, st>>>((const FusedOuterArgs<T>*)args, cstart, F);
    return cuda_error(cudaGetLastError(), "batched outer sums launch");
  }

  // The outer resamplings and statistics of F filters of this precision in one launch.
  static dpf_status scan_batch(const void* args, const int* cstart, int nctas, int F, cudaStream_t st) {
    outer_scatter_batch_kernel<T><<<nctas, OF_NT, 0, st>>>((const FusedOuterArgs<T>*)args, cstart, F);
    return cuda_error(cudaGetLastError(), "batched outer resample launch");
  }

  // The bootstrap particle filter's step t (M = 1: the state slots hold one particle a
  // group): propagation from the ancestors and the likelihood weights.
  static dpf_status pf_step(Ctx& x) {
    const long long t = x.t + 1;
    PFArgs<T> a{};
    const int so = (int)((t + 1) % 2), sn = (int)(t % 2);  // slot of step t-1 (t = 1: 0), of step t
    a.x_old = (const T*)x.x[so];
    a.z_old = (const T*)x.z[so];
    a.x_new = (T*)x.x[sn];
    a.z_new = (T*)x.z[sn];
    a.lw = (T*)x.lw;
    a.xm = (T*)x.xm;
    a.zm = (T*)x.zm;
    a.anc = x.anc;
    a.y = (const T*)x.yb + (t % 2) * x.dy;
    a.lwmax_key = x.lwmax_key;
    a.Csum = x.Csum;
    a.N = x.N;
    a.xp = x.xp;
    a.t = (uint32_t)t;
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    const HostModel& h = x.hm;
    a.gcos = h.growth ? (T)(h.gc * std::cos(h.gw * (double)(t - 1))) : T(0);
    a.first = t == 1 ? 1 : 0;
    const unsigned blocks = (unsigned)std::min<long long>((x.N + 255) / 256, 152 * 8);
    if (use_xz(x))
      pf_kernel<T, D1, D2, DY, true><<<blocks, 256, 0, x.stream>>>(cst(x), a);
    else
      pf_kernel<T, D1, D2, DY, false><<<blocks, 256, 0, x.stream>>>(cst(x), a);
    return cuda_error(cudaGetLastError(), "particle filter step launch");
  }

  // The DPF without look-ahead, call t (one CTA a group of M inner particles).
  static dpf_status std_step(Ctx& x) {
    const long long t = x.t + 1;
    StdArgs<T> a{};
    const int so = (int)((t + 1) % 2), sn = (int)(t % 2);
    a.x_old = (const T*)x.x[so];
    a.z_old = (const T*)x.z[so];
    a.lq_old = (const T*)x.lq[so];
    a.x_new = (T*)x.x[sn];
    a.z_new = (T*)x.z[sn];
    a.lq_new = (T*)x.lq[sn];
    a.lw = (T*)x.lw;
    a.xm = (T*)x.xm;
    a.zm = (T*)x.zm;
    a.anc = x.anc;
    a.y = (const T*)x.yb + (t % 2) * x.dy;
    a.lwmax_key = x.lwmax_key;
    a.Csum = x.Csum;
    a.err = x.err;
    a.N = x.N;
    a.M = x.M;
    a.xp = x.xp;
    a.t = (uint32_t)t;
    a.key = Key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    const HostModel& h = x.hm;
    a.gcos = h.growth ? (T)(h.gc * std::cos(h.gw * (double)(t - 1))) : T(0);
    a.scaleM = (T)std::ldexp(1.0, 31 - ceil_log2_i(x.M));
    a.logM = (T)std::log((double)x.M);
    a.first = t == 1 ? 1 : 0;
    a.gauss = x.std_gauss ? 1 : 0;
    a.dbg_b = x.debug ? x.dbg_b : nullptr;
    a.dbg_j = x.debug ? x.dbg_j : nullptr;
    const int nt = (x.M + 31) / 32 * 32;
    const size_t sm = sizeof(T) * (size_t)D2 * x.M + 4 * (size_t)(x.M + 1) + sizeof(T) * 32 + 4 * 64 + 16;
    const unsigned blocks = (unsigned)std::min<long long>(x.N, 152 * 8);
    auto k = use_xz(x) ? std_dpf_kernel<T, D1, D2, DY, true> : std_dpf_kernel<T, D1, D2, DY, false>;
    if (sm > 48 * 1024) {
      cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return cuda_error(e, "cudaFuncSetAttribute");
    }
    k<<<blocks, nt, sm, x.stream>>>(cst(x), a);
    return cuda_error(cudaGetLastError(), "DPF step launch");
  }

  static Variant make(int prec) {
    Variant v;
    v.pf_step = &pf_step;
    v.std_step = &std_step;
    v.xpad = &xpad;
    v.prec = prec;
    v.d1 = D1;
    v.d2 = D2;
    v.dy = DY;
    v.make_const = &make_const;
    v.init = &init;
    v.step = &step;
    v.outer = &outer;
    v.outer_args = &outer_args;
    v.outer_batch = &outer_batch;
    v.scan_batch = &scan_batch;
    v.outer_ctas = &outer_ctas;
    v.single_launch = &single_launch;
    v.oargs_size = sizeof(FusedOuterArgs<T>);
    v.step_smem = &smem;
    v.batch_args = &batch_args;
    v.region_bytes = &region_bytes;
    v.batch_launch = &batch_launch;
    v.use_xz = &use_xz;
    v.ppl_for = &ppl_for;
    v.args_size = sizeof(StepArgs<T>);
    v.const_size = sizeof(Const);
    return v;
  }
};

}  // namespace dpf
