// FP32 SIPG level operator on cells of N = 4 (the multigrid smoother's
// operator at k_p = 3, Secs. 3.2 and 3.3 of arXiv:1802.01439) with its data
// staged in shared memory by the tensor memory accelerator.
//
// Persistent warps, each working through chunks of 8 consecutive cells of one
// x-row (so the mesh needs nx divisible by 8).  For a chunk the operator
// needs the chunk itself and, because the 8 cells share y and z, four more
// contiguous 8-cell ranges: the +y, -y, +z and -z neighbours; the x-neighbours
// lie in the chunk but for the two end cells, whose outer neighbours are
// copied cell by cell.  Lane 0 of the warp issues these copies (plus the
// epilogue's b and previous iterate) as 2D tensor copies of 32 rows x 64
// bytes, completing on an mbarrier, so the loads are in flight without
// holding registers.  With one stage per warp (15 KB, 12 warps per SM) the
// lanes read the chunk into registers and the warp refills the stage with its
// next chunk at once, so the copy overlaps the whole arithmetic of the
// current chunk; with two stages (7 warps) the refill runs two chunks ahead.
// The 64-byte swizzle of the copies makes the lanes' reads of their own
// 64-byte plane conflict-free (lane 4 g + z reads row 4 g + z; its 16-byte
// quarter q sits at q ^ ((row >> 1) & 3)).  The arithmetic is that of the
// register kernel (k_plane_core.cuh).
//
// Every wait on an mbarrier is bounded; a warp whose wait gives up counts it
// in a device counter (laplace_tma_timeouts), waits (bounded) for its other
// stage and leaves.
#include <cuda.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "k_plane_core.cuh"

namespace dgns {
namespace {

using plane::Epi;
using plane::Tab;
using plane::Tab2;
using plane::XNb;

constexpr int CHUNK = 8;                 // cells per chunk
constexpr int ARR = 2048;                // bytes of one vector over a chunk
constexpr int STAGE = 15 * 1024;         // 7 vectors + the two end neighbours, 1024-aligned
constexpr int EDGE = 7 * ARR;            // offset of the end neighbours (unswizzled)
enum { A_X = 0, A_YP = 1, A_YM = 2, A_ZP = 3, A_ZM = 4, A_B = 5, A_P = 6 };
constexpr int WAIT_LIMIT = 1 << 22;      // polls of try_wait before a wait gives up

__device__ unsigned int g_tma_timeouts;

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void bar_init(uint32_t bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void bar_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool bar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < WAIT_LIMIT; ++i)
    if (bar_try(bar, parity)) return true;
  return false;
}

// 32 rows of 64 bytes starting at `row` of the vector behind `map`.
__device__ __forceinline__ void copy_rows(uint32_t dst, const CUtensorMap* map, int row, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
      "[%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(row), "r"(bar)
      : "memory");
}

__device__ __forceinline__ void copy_bytes(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

// Plane `row` of a swizzled 32-row chunk buffer.
__device__ __forceinline__ void read_plane(const unsigned char* buf, int row, float (&v)[16]) {
  const unsigned char* r = buf + row * 64;
  const int sw = (row >> 1) & 3;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 t = *reinterpret_cast<const float4*>(r + 16 * (q ^ sw));
    v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
  }
}

// Plane z of an unswizzled cell (256 bytes).
__device__ __forceinline__ void read_cell_plane(const unsigned char* cell, int z, float (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float4 t = *reinterpret_cast<const float4*>(cell + 64 * z + 16 * q);
    v[4 * q] = t.x, v[4 * q + 1] = t.y, v[4 * q + 2] = t.z, v[4 * q + 3] = t.w;
  }
}

struct Maps {
  CUtensorMap x, b, p;
};

// Lane 0: the copies of chunk q into the stage at `buf`, completing on `bar`.
// nepi: epilogue vectors to stage (0, b, or b and the previous iterate).
__device__ __forceinline__ void issue(uint32_t buf, uint32_t bar, long long q, const Maps& mp, const MeshDims& m,
                                      const float* src, bool ends, int nepi) {
  const long long c0 = q * CHUNK;
  const CellXYZ a = cell_xyz((unsigned)c0, m);
  const long long cf = (long long)a.comp * m.E;
  bar_expect(bar, (uint32_t)((5 + nepi) * ARR + (ends ? 2 * 256 : 0)));
  copy_rows(buf + A_X * ARR, &mp.x, (int)(4 * c0), bar);
  copy_rows(buf + A_YP * ARR, &mp.x, (int)(4 * (cf + neighbor32<1>(a, +1, m))), bar);
  copy_rows(buf + A_YM * ARR, &mp.x, (int)(4 * (cf + neighbor32<1>(a, -1, m))), bar);
  copy_rows(buf + A_ZP * ARR, &mp.x, (int)(4 * (cf + neighbor32<2>(a, +1, m))), bar);
  copy_rows(buf + A_ZM * ARR, &mp.x, (int)(4 * (cf + neighbor32<2>(a, -1, m))), bar);
  if (nepi >= 1) copy_rows(buf + A_B * ARR, &mp.b, (int)(4 * c0), bar);
  if (nepi >= 2) copy_rows(buf + A_P * ARR, &mp.p, (int)(4 * c0), bar);
  if (ends) {
    const CellXYZ e = cell_xyz((unsigned)(c0 + CHUNK - 1), m);
    copy_bytes(buf + EDGE, src + (size_t)(cf + neighbor32<0>(a, -1, m)) * 64, 256, bar);
    copy_bytes(buf + EDGE + 256, src + (size_t)(cf + neighbor32<0>(e, +1, m)) * 64, 256, bar);
  }
}

template <int EPI, int ZF, bool PK, int WARPS, int STAGES>
__global__ void __launch_bounds__(WARPS * 32, 1)
    sipg_tma_kernel(const __grid_constant__ Maps mp, const float* __restrict__ src, float* __restrict__ dst,
                    const __grid_constant__ Tab tb, const __grid_constant__ Tab2 tp, const MeshDims m,
                    const long long nchunks, const Epi ea) {
  unsigned char* smem = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(dyn_smem()) + 1023) & ~static_cast<uintptr_t>(1023));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, z = lane & 3;
  unsigned char* wbuf = smem + (size_t)warp * STAGES * STAGE;
  const uint32_t sbuf = smem_addr(wbuf);
  const uint32_t bar = smem_addr(smem + (size_t)WARPS * STAGES * STAGE + 16 * warp);   // one barrier per stage
  const long long nw = (long long)gridDim.x * WARPS;
  const long long w0 = (long long)blockIdx.x * WARPS + warp;
  // the end cells of a chunk have their outer x-neighbour in the chunk only
  // when the chunk is the whole x-row
  const bool ends = m.nx > CHUNK;
  const bool hasp = EPI == EPI_CHEB && ea.xprev != nullptr && ea.c1 != 0.f;
  const int nepi = EPI == EPI_NONE ? 0 : (hasp ? 2 : 1);
  if (lane == 0) {
    for (int s = 0; s < STAGES; ++s) bar_init(bar + 8 * s);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    for (int s = 0; s < STAGES; ++s)
      if (w0 + s * nw < nchunks) issue(sbuf + s * STAGE, bar + 8 * s, w0 + s * nw, mp, m, src, ends, nepi);
  }
  __syncwarp();
  float D[16];
  if constexpr (EPI == EPI_CHEB) plane::load_plane(ea.dinv + z * 16, D);
  // x-neighbours inside the chunk: lanes of cells g +- 1 (cyclic in the chunk,
  // which is right for the end cells only when the chunk is the whole row)
  const int sp = 4 * ((g + 1) & 7) + z, sm = 4 * ((g + 7) & 7) + z;
  const bool outp = ends && g == CHUNK - 1, outm = ends && g == 0;
  int k = 0;
  for (long long q = w0; q < nchunks; q += nw, ++k) {
    const int s = STAGES == 1 ? 0 : (k & 1);
    const uint32_t parity = (uint32_t)(STAGES == 1 ? k : (k >> 1)) & 1u;
    const bool ok = __all_sync(plane::FULL, bar_wait(bar + 8 * s, parity));
    if (!ok) {
      if (lane == 0) atomicAdd(&g_tma_timeouts, 1u);
      // the other stage may still have copies in flight
      if (STAGES == 2 && q + nw < nchunks) bar_wait(bar + 8 * (s ^ 1), (uint32_t)((k + 1) >> 1) & 1u);
      return;
    }
    const unsigned char* buf = wbuf + s * STAGE;
    float X[16], YP[16], YM[16], ZP[16], ZM[16];
    read_plane(buf + A_X * ARR, lane, X);
    read_plane(buf + A_YP * ARR, lane, YP);
    read_plane(buf + A_YM * ARR, lane, YM);
    read_plane(buf + A_ZP * ARR, lane, ZP);
    read_plane(buf + A_ZM * ARR, lane, ZM);
    XNb n;
    plane::xnb_shuffle(tb, X, sp, sm, n);
    if (outp) {
      float P[16];
      read_cell_plane(buf + EDGE + 256, z, P);
      plane::xnb_from_plane(tb, P, +1, n);
    }
    if (outm) {
      float P[16];
      read_cell_plane(buf + EDGE, z, P);
      plane::xnb_from_plane(tb, P, -1, n);
    }
    float B[16], P[16];
    if constexpr (EPI != EPI_NONE) read_plane(buf + A_B * ARR, lane, B);
    if (hasp) read_plane(buf + A_P * ARR, lane, P);
    // the stage is free once every lane has read it: refill it STAGES chunks
    // ahead (with one stage, the copy overlaps this chunk's arithmetic)
    __syncwarp();
    if (lane == 0 && q + STAGES * nw < nchunks) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue(sbuf + s * STAGE, bar + 8 * s, q + STAGES * nw, mp, m, src, ends, nepi);
    }
    float O[16];
    if constexpr (PK) {
      float2 Y[8];
      plane::apply2<ZF>(tb, tp, z, X, n, YP, YM, ZP, ZM, Y);
      plane::epilogue2<EPI>(ea, X, Y, B, D, P, hasp, O);
    } else {
      float Y[16];
      plane::apply<ZF>(tb, z, X, n, YP, YM, ZP, ZM, Y);
      plane::epilogue<EPI>(ea, X, Y, B, D, P, hasp, O);
    }
    plane::store_plane(dst + (size_t)(q * CHUNK + g) * 64 + z * 16, O);
  }
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiled encoder() {
  static EncodeTiled fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  });
  return fn;
}

// A vector of nrows 64-byte planes as a 2D tensor (16 floats x nrows), read
// in boxes of 32 rows with the 64-byte swizzle.
bool encode(CUtensorMap* map, const float* base, long long nrows) {
  EncodeTiled fn = encoder();
  if (!fn || base == nullptr) return false;
  const cuuint64_t dims[2] = {16, (cuuint64_t)nrows};
  const cuuint64_t strides[1] = {64};
  const cuuint32_t box[2] = {16, 32};
  const cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int WARPS, int STAGES>
constexpr size_t tma_smem() {
  return (size_t)WARPS * STAGES * STAGE + 16 * WARPS + 1024;
}

template <int EPI, int ZF, bool PK, int WARPS, int STAGES>
int launch_tma(const Maps& mp, const MeshDims& m, long long nchunks, const float* src, float* dst, const Tab& tb,
               const Tab2& tp, const Epi& ea, cudaStream_t s) {
  static std::atomic<int> attr_dev{-1};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 2;
  if (attr_dev.load() != dev) {
    if (cudaFuncSetAttribute(sipg_tma_kernel<EPI, ZF, PK, WARPS, STAGES>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)tma_smem<WARPS, STAGES>()) != cudaSuccess)
      return 2;
    attr_dev.store(dev);
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 2;
  long long blocks = (nchunks + WARPS - 1) / WARPS;
  if (blocks > sms) blocks = sms;
  sipg_tma_kernel<EPI, ZF, PK, WARPS, STAGES><<<(unsigned)blocks, WARPS * 32, tma_smem<WARPS, STAGES>(), s>>>(mp, src, dst, tb, tp,
                                                                                              m, nchunks, ea);
  return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

template <int ZF, bool PK, int WARPS, int STAGES>
int launch_tma_epi(int epi, const Maps& mp, const MeshDims& m, long long nchunks, const float* src, float* dst,
                   const Tab& tb, const Tab2& tp, const Epi& ea, cudaStream_t s) {
  switch (epi) {
    case EPI_NONE: return launch_tma<EPI_NONE, ZF, PK, WARPS, STAGES>(mp, m, nchunks, src, dst, tb, tp, ea, s);
    case EPI_RESID: return launch_tma<EPI_RESID, ZF, PK, WARPS, STAGES>(mp, m, nchunks, src, dst, tb, tp, ea, s);
    case EPI_CHEB: return launch_tma<EPI_CHEB, ZF, PK, WARPS, STAGES>(mp, m, nchunks, src, dst, tb, tp, ea, s);
  }
  return 1;
}

bool aligned32(const void* p) { return p == nullptr || (reinterpret_cast<uintptr_t>(p) & 31) == 0; }

}  // namespace

int laplace_tma_f32(const MeshDims& m, int ncomp, const float* src, float* dst, const LapHost& h, int epi,
                    const EpiHost& eh, cudaStream_t s, int variant) {
  if (h.N != 4 || m.nx % CHUNK != 0) return -1;
  if (!aligned32(src) || !aligned32(dst) || !aligned32(eh.b) || !aligned32(eh.xprev) || !aligned32(eh.dinv))
    return -1;
  const long long ncells = m.E * ncomp;
  if (ncells == 0) return 0;
  const long long nrows = 4 * ncells;
  if (nrows > 0x7fffffffLL) return -1;
  Maps mp;
  if (!encode(&mp.x, src, nrows)) return -1;
  mp.b = mp.x;
  mp.p = mp.x;
  if (epi != EPI_NONE && !encode(&mp.b, (const float*)eh.b, nrows)) return -1;
  if (epi == EPI_CHEB && eh.xprev && !encode(&mp.p, (const float*)eh.xprev, nrows)) return -1;
  Tab tb;
  plane::make_tab(h, tb);
  Tab2 tp;
  plane::make_tab2(tb, tp);
  const Epi ea{(const float*)eh.b, (const float*)eh.xprev, (const float*)eh.dinv, (float)eh.c1, (float)eh.c2};
  const long long nchunks = ncells / CHUNK;
  switch (variant) {
    case 0: return launch_tma_epi<1, true, 12, 1>(epi, mp, m, nchunks, src, dst, tb, tp, ea, s);
    case 1: return launch_tma_epi<1, true, 7, 2>(epi, mp, m, nchunks, src, dst, tb, tp, ea, s);
  }
  return -1;
}

unsigned laplace_tma_timeouts() {
  unsigned v = 0;
  if (cudaMemcpyFromSymbol(&v, g_tma_timeouts, sizeof(v)) != cudaSuccess) return ~0u;
  return v;
}

}  // namespace dgns
