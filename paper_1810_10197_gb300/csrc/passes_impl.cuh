// Launchers for the five passes: pick the kernel instantiation for the run-time line length
// and size the grid and the dynamic shared memory.
#pragma once

#include "passes.cuh"
#include "zpass_rr.cuh"
#include "ypass_tma.cuh"
#include "xpass_tma.cuh"

namespace dns {

template <typename K>
static cudaError_t set_smem(K kernel, size_t bytes) {
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Persistent grid: as many CTAs as the device holds at once (at most one per tile).
template <typename K>
static cudaError_t persistent_grid(K kernel, int threads, size_t smem, long long tiles, unsigned* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long cap = (long long)sms * per_sm;
  *grid = (unsigned)(tiles < cap ? (tiles > 0 ? tiles : 1) : cap);
  return cudaSuccess;
}

static cudaError_t launch_p1_tma(const PassArgs& a, cudaStream_t s);
template <typename T, int N, bool B>
static cudaError_t launch_p1(const PassArgs& a, cudaStream_t s) {
  using V = v2_t<T>;
  if constexpr (std::is_same<T, float>::value && N == 256 && !B) {
    if (x_tma_applies(a)) {
      // a driver without tensor-map encoding (or a view it refuses) runs the shared-memory kernel
      const cudaError_t e = launch_p1_tma(a, s);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  constexpr int TC = p1_cols<T, N>();
  const size_t smem = (size_t)(twiddle_count_xy(N) + 3 * TC * line_ld<V, N>()) * sizeof(V) +
                      (size_t)2 * TC * sizeof(T);
  cudaError_t e = set_smem(k_p1<T, N, B>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.g.MyMz + TC / 2 - 1) / (TC / 2), B ? 2 : 1);
  k_p1<T, N, B><<<grid, FftPlan<N>::G * 3 * TC, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, bool B>
static cudaError_t launch_p5(const PassArgs& a, cudaStream_t s) {
  using V = v2_t<T>;
  constexpr int TC = p5_cols<T, N>(B);
  constexpr int NF = B ? 6 : 3;
  const size_t smem = (size_t)(twiddle_count_xy(N) + NF * TC * line_ld<V, N>()) * sizeof(V) +
                      (size_t)(a.g.Mx + TC) * sizeof(double) + (size_t)2 * TC * sizeof(T);
  cudaError_t e = set_smem(k_p5<T, N, B>, smem);
  if (e != cudaSuccess) return e;
  dim3 grid((a.g.MyMz + TC - 1) / TC);
  k_p5<T, N, B><<<grid, FftPlan<N>::G * NF * TC, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, bool INV, int VAR>
static cudaError_t launch_py_v(const PassArgs& a, cudaStream_t s) {
  using V = v2_t<T>;
  constexpr int TZ = py_cols<T, VAR>();
  const size_t smem = (size_t)(twiddle_count_xy(N) + TZ * line_ld<V, N>()) * sizeof(V);
  cudaError_t e = set_smem(k_py<T, N, INV, VAR>, smem);
  if (e != cudaSuccess) return e;
  const int nf = INV ? (a.g.bouss ? 7 : 6) : (a.g.bouss ? 6 : 3);
  dim3 grid((a.g.Mz + TZ - 1) / TZ, a.g.nx, nf);
  k_py<T, N, INV, VAR><<<grid, FftPlan<N>::G * TZ, smem, s>>>(a);
  return cudaGetLastError();
}
// y-pass variant 2: tensor-map tile copies and register-resident transforms (FP32,
// ny = 256, Mz even); elsewhere it runs variant 0.  The tensor maps are encoded on the host
// for every launch (they hold the buffer addresses; a captured graph keeps them by value).
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      (void)cudaGetLastError();   // not sticky: leave no error for the launch checks that follow
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}
// FP32 view [planes][rows][2 Mz] of a pass buffer, box {2 cols, rows, 1} (cols complex columns
// of every row of one plane: 8 or 16, with the 64- or 128-byte swizzle), zero fill outside
static cudaError_t plane_map(CUtensorMap* m, const void* p, int Mz, int rows, long long planes, int cols = 8) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dim[3] = {(cuuint64_t)(2 * Mz), (cuuint64_t)rows, (cuuint64_t)planes};
  const cuuint64_t stride[2] = {(cuuint64_t)Mz * 8, (cuuint64_t)rows * Mz * 8};
  const cuuint32_t box[3] = {(cuuint32_t)(2 * cols), (cuuint32_t)rows, 1};
  const cuuint32_t estride[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<void*>(p), dim, stride, box, estride,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, cols == 16 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorNotSupported;
}
// x-inverse pass with tensor-map tile copies: grid ceil(MyMz / 8).
template <bool Y32>
static cudaError_t launch_p1_tma_t(const PassArgs& a, cudaStream_t s) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const int MyMz = a.g.MyMz, Mx = a.g.Mx;
  CUtensorMap ty[2], tout;
  for (int i = 0; i < 2; ++i) {
    const void* p = a.ycand[i] ? a.ycand[i] : a.ycand[0];
    const cuuint64_t dim[3] = {(cuuint64_t)(2 * MyMz), (cuuint64_t)Mx, 3};
    const cuuint64_t stride[2] = {(cuuint64_t)MyMz * (Y32 ? 8 : 16), (cuuint64_t)Mx * MyMz * (Y32 ? 8 : 16)};
    const cuuint32_t box[3] = {16, (cuuint32_t)Mx, 1};
    const cuuint32_t estride[3] = {1, 1, 1};
    if (enc(&ty[i], Y32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<void*>(p), dim,
            stride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE,
            Y32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorNotSupported;
  }
  cudaError_t e = plane_map(&tout, a.out, MyMz, a.g.nx, 6);
  if (e != cudaSuccess) return e;
  const size_t smem = xtma_p1_smem(Mx, Y32);
  if ((e = set_smem(k_p1_tma<256, Y32>, smem)) != cudaSuccess) return e;
  PassArgs b = a;
  if (!b.ycand[1]) b.ycand[1] = b.ycand[0];
  k_p1_tma<256, Y32><<<(MyMz + 7) / 8, 128, smem, s>>>(b, ty[0], ty[1], tout);
  return cudaGetLastError();
}
static cudaError_t launch_p1_tma(const PassArgs& a, cudaStream_t s) {
  return a.ycand_f32 ? launch_p1_tma_t<true>(a, s) : launch_p1_tma_t<false>(a, s);
}
template <int N, bool INV>
static cudaError_t launch_py_tma(const PassArgs& a, cudaStream_t s) {
  constexpr int TZ = YtmaTile<N>::TZ;
  const int nf = INV ? (a.g.bouss ? 7 : 6) : (a.g.bouss ? 6 : 3);
  const long long planes = (long long)nf * a.g.nx;
  CUtensorMap tin, tout;
  cudaError_t e = plane_map(&tin, a.in, a.g.Mz, INV ? a.g.My : a.g.ny, planes, TZ);
  if (e != cudaSuccess) return e;
  if ((e = plane_map(&tout, a.out, a.g.Mz, INV ? a.g.ny : a.g.My, planes, TZ)) != cudaSuccess) return e;
  const size_t smem = ytma_smem<N, INV>();
  if ((e = set_smem(k_py_tma<N, INV>, smem)) != cudaSuccess) return e;
  dim3 grid((a.g.Mz + TZ - 1) / TZ, a.g.nx, nf);
  k_py_tma<N, INV><<<grid, 128, smem, s>>>(a, tin, tout);
  return cudaGetLastError();
}
template <typename T, int N, bool INV>
static cudaError_t launch_py(const PassArgs& a, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value && (N == 256 || N == 128)) {
    if (a.var_py == 2 && ytma_supported(a.g.ny, a.g.Mz)) {
      // a driver without tensor-map encoding (or a view it refuses) runs variant 0
      const cudaError_t e = launch_py_tma<N, INV>(a, s);
      if (e != cudaErrorNotSupported) return e;
    }
  }
  return a.var_py == 1 ? launch_py_v<T, N, INV, 1>(a, s) : launch_py_v<T, N, INV, 0>(a, s);
}

template <typename T, int MZ, bool B, int VAR>
static cudaError_t launch_p3_v(const PassArgs& a, cudaStream_t s) {
  using V = v2_t<T>;
  constexpr int TL = p3_lines<T, MZ, B, VAR>();
  constexpr int NIN = B ? 7 : 6;
  const size_t lines_elems = (size_t)twiddle_count_z(2 * MZ) + NIN * TL * p3_ld<V, MZ>();
  size_t smem = lines_elems * sizeof(V);
  // bulk path: staging rows and the mbarrier, when a row is a multiple of 16 bytes and the
  // whole fits in a CTA's shared memory
  const size_t smem_bulk = p3_stage_offset<V>(lines_elems) + (size_t)NIN * TL * a.g.Mz * sizeof(V) + 16;
  PassArgs b = a;
  b.p3_bulk = a.p3_bulk && (a.g.Mz * sizeof(V)) % 16 == 0 && smem_bulk <= 232448;
  if (!b.p3_bulk) b.p3_stall = 0;
  if (b.p3_bulk) smem = smem_bulk;
  cudaError_t e = set_smem(k_p3<T, MZ, B, VAR>, smem);
  if (e != cudaSuccess) return e;
  const long long nxy = (long long)a.g.nx * a.g.ny;
  dim3 grid((unsigned)((nxy + TL - 1) / TL));
  k_p3<T, MZ, B, VAR><<<grid, FftPlan<MZ>::G * NIN * TL, smem, s>>>(b);
  return cudaGetLastError();
}
// The register-resident FP32 z pass: persistent CTAs of 128 threads, as many as fit on the
// device at once; the tile variant selects fully paired (0) or paired-sum / scalar-product
// (1) FP32 arithmetic.
template <int N, bool PAIRED>
static cudaError_t launch_p3_rr_v(const PassArgs& a, cudaStream_t s) {
  const size_t smem = zrr_smem<N>(a.g.Mz);
  cudaError_t e = set_smem(k_p3_rr<N, PAIRED>, smem);
  if (e != cudaSuccess) return e;
  const long long nxy = (long long)a.g.nx * a.g.ny;
  const long long tiles = (nxy + ZrrPlan<N, 128>::TL - 1) / ZrrPlan<N, 128>::TL;
  unsigned grid = 0;
  if ((e = persistent_grid(k_p3_rr<N, PAIRED>, 128, smem, tiles, &grid)) != cudaSuccess) return e;
  k_p3_rr<N, PAIRED><<<grid, 128, smem, s>>>(a);
  return cudaGetLastError();
}
template <int N>
static cudaError_t launch_p3_rr(const PassArgs& a, cudaStream_t s) {
  return a.var_p3 ? launch_p3_rr_v<N, false>(a, s) : launch_p3_rr_v<N, true>(a, s);
}

template <typename T, int MZ, bool B>
static cudaError_t launch_p3(const PassArgs& a, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value && !B && zrr_supported(2 * MZ)) {
    if (p3_rr_applies(a)) return launch_p3_rr<2 * MZ>(a, s);
  }
  return a.var_p3 ? launch_p3_v<T, MZ, B, 1>(a, s) : launch_p3_v<T, MZ, B, 0>(a, s);
}

#define DNS_XY_SIZES(X) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768)
#define DNS_ZH_SIZES(X) X(4) X(6) X(8) X(12) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384)
// the double-word form: lines of 32 points and more (its kernels are large; every
// instantiation costs seconds of compile time)
#define DNS_XY_SIZES_DW(X) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384) X(512) X(768)
#define DNS_ZH_SIZES_DW(X) X(16) X(24) X(32) X(48) X(64) X(96) X(128) X(192) X(256) X(384)

// Pass WHICH (1..5) for element type T; cudaErrorInvalidValue for an unsupported line length.
template <typename T, int WHICH>
cudaError_t launch_pass_w(const PassArgs& a, cudaStream_t s) {
  if constexpr (is_dw<T>()) {
    if constexpr (WHICH == 1 || WHICH == 5) {
      switch (a.g.nx) {
#define CD(N)                                                                           \
  case N:                                                                               \
    if (WHICH == 1) return a.g.bouss ? launch_p1<T, N, true>(a, s) : launch_p1<T, N, false>(a, s); \
    return a.g.bouss ? launch_p5<T, N, true>(a, s) : launch_p5<T, N, false>(a, s);
        DNS_XY_SIZES_DW(CD)
#undef CD
      }
    } else if constexpr (WHICH == 2 || WHICH == 4) {
      switch (a.g.ny) {
#define CD(N) case N: return launch_py<T, N, WHICH == 2>(a, s);
        DNS_XY_SIZES_DW(CD)
#undef CD
      }
    } else {
      switch (a.g.nz / 2) {
#define CD(N) case N: return a.g.bouss ? launch_p3<T, N, true>(a, s) : launch_p3<T, N, false>(a, s);
        DNS_ZH_SIZES_DW(CD)
#undef CD
      }
    }
    return cudaErrorInvalidValue;
  } else {
    if constexpr (WHICH == 1) {
      switch (a.g.nx) {
#define C1(N) case N: return a.g.bouss ? launch_p1<T, N, true>(a, s) : launch_p1<T, N, false>(a, s);
        DNS_XY_SIZES(C1)
#undef C1
      }
    } else if constexpr (WHICH == 2) {
      switch (a.g.ny) {
#define C2(N) case N: return launch_py<T, N, true>(a, s);
        DNS_XY_SIZES(C2)
#undef C2
      }
    } else if constexpr (WHICH == 3) {
      switch (a.g.nz / 2) {
#define C3(N) case N: return a.g.bouss ? launch_p3<T, N, true>(a, s) : launch_p3<T, N, false>(a, s);
        DNS_ZH_SIZES(C3)
#undef C3
      }
    } else if constexpr (WHICH == 4) {
      switch (a.g.ny) {
#define C4(N) case N: return launch_py<T, N, false>(a, s);
        DNS_XY_SIZES(C4)
#undef C4
      }
    } else {
      switch (a.g.nx) {
#define C5(N) case N: return a.g.bouss ? launch_p5<T, N, true>(a, s) : launch_p5<T, N, false>(a, s);
        DNS_XY_SIZES(C5)
#undef C5
      }
    }
    return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_pass(int which, const PassArgs& a, cudaStream_t s) {
  switch (which) {
    case 1: return launch_pass_w<T, 1>(a, s);
    case 2: return launch_pass_w<T, 2>(a, s);
    case 3: return launch_pass_w<T, 3>(a, s);
    case 4: return launch_pass_w<T, 4>(a, s);
    case 5: return launch_pass_w<T, 5>(a, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dns
