// Launchers of a variant whose model constants are too large for a launch
// parameter (a z block of a few tens of coordinates): the block kernel only,
// the constants in device memory, models whose x transition is free of z, and
// the propagation A_zz z on the tensor cores (3xTF32) when the shapes allow it
// (FP32, M = 128 or 256, d2 % 8 == 0).
#pragma once

#include "dpf_variant.cuh"

namespace dpf {

// The step launch of a wide variant (x transition free of z), with or without
// the tensor-core propagation; each is instantiated in a translation unit of its
// own (dpf_wide_launch.cuh), so that the two large kernels compile in parallel.
template <typename T, int D1, int D2, int DY, bool TC>
dpf_status wide_launch(Ctx& x, StepArgs<T>& a, cudaStream_t s);

template <typename T, int D1, int D2, int DY>
struct WideVariantImpl {
  typedef VariantImpl<T, D1, D2, DY, 0> Base;
  typedef MC<T, D1, D2, DY> Const;
  static constexpr int MAX_M = 256;  // one inner particle a thread

  static bool tc_shape(int M) { return sizeof(T) == 4 && D2 % 8 == 0 && (M == 128 || M == 256); }

  static size_t smem(int M, int L, bool, int) {
    return step_geometry<T, D1, D2, DY, false>(M, L, threads_for(M), nullptr, false, 1, tc_shape(M));
  }

  static dpf_status upload(Ctx& x) {
    if (x.d_mconst) return DPF_OK;
    cudaError_t e = cudaMalloc(&x.d_mconst, sizeof(Const));
    if (e != cudaSuccess) {
      x.d_mconst = nullptr;
      return cuda_error(e, "model constants");
    }
    x.allocs.push_back(x.d_mconst);
    // x.mconst (host) lives as long as the context
    e = cudaMemcpyAsync(x.d_mconst, x.mconst.data(), sizeof(Const), cudaMemcpyHostToDevice, x.stream);
    return cuda_error(e, "model constants upload");
  }

  static dpf_status init(Ctx& x) {
    dpf_status st = upload(x);
    if (st) return st;
    const Key key{(uint32_t)x.seed, (uint32_t)(x.seed >> 32)};
    init_kernel_g<T, D1, D2, DY><<<(unsigned)x.N, threads_for(x.M), 0, x.stream>>>(
        (const Const*)x.d_mconst, (T*)x.z[0], (T*)x.lq[0], (T*)x.x[0], x.N, x.M, x.xp, key);
    return cuda_error(cudaGetLastError(), "init kernel launch");
  }

  static dpf_status launch(Ctx& x, StepArgs<T>& a, cudaStream_t s) {
    return x.tensor_cores && tc_shape(x.M) ? wide_launch<T, D1, D2, DY, true>(x, a, s)
                                           : wide_launch<T, D1, D2, DY, false>(x, a, s);
  }

  static dpf_status step(Ctx& x, int) {
    StepArgs<T> a{};
    Base::fill_args(x, a);
    return launch(x, a, x.stream);
  }

  // A batched member's step (its own launch, on the batch's stream s) from the
  // arguments batch_args filled with the batch's observation rows.
  static void batch_args(Ctx& x, const void* y_prev, const void* y_cur, bool, void* out) {
    StepArgs<T> a{};
    Base::fill_args(x, a);
    a.y_prev = (const T*)y_prev;
    a.y_cur = (const T*)y_cur;
    memcpy(out, &a, sizeof(a));
  }
  static dpf_status single_launch(Ctx& x, const void* args, int, bool, cudaStream_t s) {
    StepArgs<T> a;
    memcpy(&a, args, sizeof(a));
    return launch(x, a, s);
  }

  static Variant make(int prec) {
    Variant v{};
    v.xpad = &Base::xpad;
    v.prec = prec;
    v.d1 = D1;
    v.d2 = D2;
    v.dy = DY;
    v.make_const = &Base::make_const;
    v.init = &init;
    v.step = &step;
    v.outer = &Base::outer;
    v.outer_args = &Base::outer_args;
    v.outer_ctas = &Base::outer_ctas;
    v.outer_batch = &Base::outer_batch;
    v.scan_batch = &Base::scan_batch;
    v.step_smem = &smem;
    // batched: one launch a filter (no shared launch for a class), all on the batch's
    // stream, since the launches share the translation unit's constant bank
    v.batch_args = &batch_args;
    v.single_launch = &single_launch;
    v.batch_serial = true;
    v.region_bytes = nullptr;
    v.batch_launch = nullptr;
    v.use_xz = &Base::use_xz;
    v.ppl_for = &Base::ppl_for;
    v.args_size = sizeof(StepArgs<T>);
    v.const_size = sizeof(Const);
    v.oargs_size = sizeof(FusedOuterArgs<T>);
    v.max_m = MAX_M;
    v.has_tc = tc_shape(256);
    v.xz_supported = false;
    return v;
  }
};

}  // namespace dpf
