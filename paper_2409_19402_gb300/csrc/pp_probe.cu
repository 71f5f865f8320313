// pp_probe.cu -- pp_peak_probe: short kernels that measure the arithmetic
// peaks the roofline of the facewise SVD and of the tensor-core products is
// quoted against (instrumentation; no counterpart in the paper).
//
// kind 0 (FP32 FMA): every thread of a full-device grid runs `reps` rounds of
// 16 independent FMA chains in registers (2 flop per FMA).
// kind 1 (tcgen05 kind::tf32): one CTA per SM issues `reps` MMAs of
// M = 128, N = 256, K = 8 (2 M N K flop each) from zeroed shared-memory
// operands into TMEM, commits them and waits (bounded) for completion.
// The caller times the call with CUDA events on `stream`; *flops receives the
// work the launch does.
#include "pp_internal.h"
#include "pp_tc.cuh"

namespace pp {
namespace {

__device__ float g_probe_sink;   // keeps the FMA chains live

constexpr int FMA_THREADS = 256, FMA_CHAINS = 16;

__global__ void __launch_bounds__(FMA_THREADS) fma_probe_kernel(int64_t reps, float seed) {
  float v[FMA_CHAINS];
#pragma unroll
  for (int q = 0; q < FMA_CHAINS; ++q) v[q] = seed + (float)(threadIdx.x + q);
  const float a = 0.999999f, b = 1e-7f;
  for (int64_t r = 0; r < reps; ++r) {
#pragma unroll
    for (int q = 0; q < FMA_CHAINS; ++q) v[q] = fmaf(v[q], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int q = 0; q < FMA_CHAINS; ++q) s += v[q];
  if (s == 12345.678f) g_probe_sink = s;   // never true for these inputs
}

constexpr int MMA_N = 256;
constexpr uint32_t MMA_IDESC = tc::tf32_idesc(128, MMA_N);

__global__ void __launch_bounds__(128) mma_probe_kernel(int64_t reps, int32_t *status) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // the 1024-byte aligned base, offset from smem_raw itself so that the
  // compiler still sees shared-memory accesses (not generic ones) through it
  unsigned char *smem = smem_raw + ((1024u - (tc::smem_u32(smem_raw) & 1023u)) & 1023u);
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_sh;
  const int tid = threadIdx.x;
  // A: 128 rows x 128 B, B: 256 rows x 128 B, zero (SW128 K-major tiles)
  for (int i = tid; i < (128 + MMA_N) * 128 / 16; i += blockDim.x)
    reinterpret_cast<float4 *>(smem)[i] = make_float4(0.f, 0.f, 0.f, 0.f);
  if (tid < 32) tc::tmem_alloc(&tmem_sh, MMA_N);
  if (tid == 0) {
    tc::mbar_init(&mbar);
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;");
  const uint32_t tmem = tmem_sh;
  if (tid == 0) {
    const uint64_t da = tc::sw128_desc(tc::smem_u32(smem));
    const uint64_t db = tc::sw128_desc(tc::smem_u32(smem + 128 * 128));
    for (int64_t r = 0; r < reps; ++r) {
      const uint64_t o = 2u * (uint32_t)(r & 3);   // walk the four K steps of the tile
      tc::mma_tf32(tmem, da + o, db + o, MMA_IDESC, r > 0 ? 1u : 0u);
    }
    tc::mma_commit(tc::smem_u32(&mbar));
  }
  __syncwarp();
  const bool ok = tc::mbar_wait(tc::smem_u32(&mbar), 0);
  if (!ok && status) atomicCAS(status, 0, PP_ETIMEOUT);
  asm volatile("tcgen05.fence::before_thread_sync;");
  __syncthreads();
  if (tid < 32) {
    asm volatile("tcgen05.fence::after_thread_sync;");
    tc::tmem_dealloc(tmem, MMA_N);
  }
}

}  // namespace
}  // namespace pp

extern "C" pp_status pp_peak_probe(int32_t kind, int64_t reps, double *flops, int32_t *status,
                                   void *stream) {
  if (reps < 1 || reps > ((int64_t)1 << 40) || !flops) return PP_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int sms = pp::num_sms();
  if (kind == 0) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pp::fma_probe_kernel,
                                                      pp::FMA_THREADS, 0) != cudaSuccess ||
        per_sm < 1)
      return PP_ECUDA;
    const int64_t blocks = (int64_t)per_sm * sms;
    pp::count_launch(1);
    pp::fma_probe_kernel<<<(unsigned)blocks, pp::FMA_THREADS, 0, st>>>(reps, 1.f);
    *flops = 2.0 * (double)blocks * pp::FMA_THREADS * pp::FMA_CHAINS * (double)reps;
    return cudaGetLastError() == cudaSuccess ? PP_OK : PP_ECUDA;
  }
  if (kind == 1) {
    const size_t smem = (size_t)(128 + pp::MMA_N) * 128 + 1024;
    if (cudaFuncSetAttribute(pp::mma_probe_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
      return PP_ECUDA;
    pp::count_launch(1);
    pp::mma_probe_kernel<<<(unsigned)sms, 128, smem, st>>>(reps, status);
    *flops = 2.0 * 128.0 * pp::MMA_N * 8.0 * (double)reps * sms;
    return cudaGetLastError() == cudaSuccess ? PP_OK : PP_ECUDA;
  }
  return PP_EINVAL;
}
