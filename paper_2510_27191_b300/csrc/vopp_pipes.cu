// Issue-rate microbenchmark of the arithmetic the leaf kernel is built from: FP32 FMA
// (scalar and packed f32x2), 32-bit integer multiply-add (low and high half of the product),
// three-input XOR, integer add, the special-function approximations (ex2, lg2, sin, sqrt,
// rsqrt) and one whole Philox4x32-10 call.  These rates bound the leaf kernel, which is
// issue-bound arithmetic rather than a memory or tensor-core workload.
//
// Each thread runs kChains dependency chains of one operation for kIters iterations (the
// integer chains are quadratic or coupled in pairs, so the compiler cannot merge steps of a
// chain), so the scheduler always has independent work; every CTA records its SM and
// the SM's cycle counter at its start and end.  The rate per SM is the operations that SM
// executed divided by the cycles between its first start and its last end, which makes the
// figure independent of the clock the SM happened to run at.  The CUDA-event duration of
// the launch gives the absolute rate at the clock of the moment.
#include <cstdint>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "vopp.h"
#include "vopp_device.cuh"
#include "vopp_internal.h"

namespace {

constexpr int kChains = 8;
constexpr int kIters = 4096;
constexpr int kThreads = 256;
constexpr int kBlocksPerSm = 4;

enum PipeOp {
  OP_FFMA, OP_FFMA2, OP_IMAD, OP_UMULHI, OP_XOR3, OP_IADD, OP_EX2, OP_LG2, OP_SIN, OP_SQRT,
  OP_RSQRT, OP_PHILOX, OP_COUNT
};

const char *const kOpNames[OP_COUNT] = {
    "fma.rn.f32", "fma.rn.f32x2", "mad.lo.u32", "mad.hi.u32", "xor3 (lop3.b32)", "add.u32",
    "ex2.approx.ftz.f32", "lg2.approx.ftz.f32", "sin.approx.ftz.f32", "sqrt.approx.ftz.f32",
    "rsqrt.approx.ftz.f32", "philox4x32-10 call"};

struct BlockClock {
  uint32_t smid;
  uint32_t pad;
  long long start, end;
};

__device__ __forceinline__ uint32_t smid() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(r));
  return r;
}

template <int OP>
__global__ void __launch_bounds__(kThreads) k_pipe(BlockClock *clocks, uint32_t *sink,
                                                   uint32_t seed) {
  __syncthreads();
  const long long t0 = clock64();
  uint32_t u[kChains];
  float f[kChains];
  unsigned long long p[kChains];   // packed f32x2 chains
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    u[c] = seed + threadIdx.x * 77u + c * 131u;
    f[c] = 0.5f + 0.01f * (float)((threadIdx.x + c) & 15);
    p[c] = ((unsigned long long)__float_as_uint(f[c]) << 32) | __float_as_uint(f[c]);
  }
  const float fm = 0.999f, fb = 1e-3f;
  const unsigned long long pm = ((unsigned long long)__float_as_uint(fm) << 32) |
                                __float_as_uint(fm);
  const unsigned long long pb = ((unsigned long long)__float_as_uint(fb) << 32) |
                                __float_as_uint(fb);
  const uint32_t um = 0x9E3779B9u, ub = 0x7F4A7C15u;
  for (int it = 0; it < kIters; ++it) {
#pragma unroll
    for (int c = 0; c < kChains; ++c) {
      if constexpr (OP == OP_FFMA) {
        asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f[c]) : "f"(fm), "f"(fb));
      } else if constexpr (OP == OP_FFMA2) {
        asm volatile("fma.rn.f32x2 %0, %0, %1, %2;" : "+l"(p[c]) : "l"(pm), "l"(pb));
      } else if constexpr (OP == OP_IMAD) {
        // x <- x*x + b: quadratic, so the compiler cannot merge steps of the chain
        asm volatile("mad.lo.u32 %0, %0, %0, %1;" : "+r"(u[c]) : "r"(ub));
      } else if constexpr (OP == OP_UMULHI) {
        // x <- hi(x * y) + m, chains coupled in pairs
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(u[c]) : "r"(u[c ^ 1]), "r"(um));
      } else if constexpr (OP == OP_XOR3) {
        // chains coupled in pairs (x ^= y ^ m, then y ^= x ^ m) so no step is loop-invariant
        asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(u[c]) : "r"(u[c ^ 1]), "r"(um));
      } else if constexpr (OP == OP_IADD) {
        asm volatile("add.u32 %0, %0, %1;" : "+r"(u[c]) : "r"(u[c ^ 1]));
      } else if constexpr (OP == OP_EX2) {
        asm volatile("ex2.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      } else if constexpr (OP == OP_LG2) {
        asm volatile("lg2.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      } else if constexpr (OP == OP_SIN) {
        asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      } else if constexpr (OP == OP_SQRT) {
        asm volatile("sqrt.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      } else if constexpr (OP == OP_RSQRT) {
        asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(f[c]));
      } else if constexpr (OP == OP_PHILOX) {
        const uint4 r = vopp::philox(make_uint4(u[c], it, c, threadIdx.x), seed, ub);
        u[c] = r.x ^ r.y ^ r.z ^ r.w;
      }
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) {
    clocks[blockIdx.x].smid = smid();
    clocks[blockIdx.x].start = t0;
    clocks[blockIdx.x].end = t1;
  }
  // every chain ends in one store per thread, so no step can be dropped or moved
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c)
    acc ^= u[c] ^ __float_as_uint(f[c]) ^ (uint32_t)p[c] ^ (uint32_t)(p[c] >> 32);
  sink[blockIdx.x * kThreads + threadIdx.x] = acc;
}

template <int OP>
cudaError_t launch_op(unsigned grid, BlockClock *clocks, uint32_t *sink, cudaStream_t s) {
  k_pipe<OP><<<grid, kThreads, 0, s>>>(clocks, sink, 0x1234567u);
  return cudaGetLastError();
}

cudaError_t launch_any(int op, unsigned grid, BlockClock *clocks, uint32_t *sink,
                       cudaStream_t s) {
  switch (op) {
    case OP_FFMA: return launch_op<OP_FFMA>(grid, clocks, sink, s);
    case OP_FFMA2: return launch_op<OP_FFMA2>(grid, clocks, sink, s);
    case OP_IMAD: return launch_op<OP_IMAD>(grid, clocks, sink, s);
    case OP_UMULHI: return launch_op<OP_UMULHI>(grid, clocks, sink, s);
    case OP_XOR3: return launch_op<OP_XOR3>(grid, clocks, sink, s);
    case OP_IADD: return launch_op<OP_IADD>(grid, clocks, sink, s);
    case OP_EX2: return launch_op<OP_EX2>(grid, clocks, sink, s);
    case OP_LG2: return launch_op<OP_LG2>(grid, clocks, sink, s);
    case OP_SIN: return launch_op<OP_SIN>(grid, clocks, sink, s);
    case OP_SQRT: return launch_op<OP_SQRT>(grid, clocks, sink, s);
    case OP_RSQRT: return launch_op<OP_RSQRT>(grid, clocks, sink, s);
    case OP_PHILOX: return launch_op<OP_PHILOX>(grid, clocks, sink, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

extern "C" VOPP_API int vopp_pipe_rates(int device, vopp_pipe_rate *out, int32_t max_out,
                                        int32_t *n_out) {
  if (!out || !n_out || max_out < 0) {
    return vopp::set_error(VOPP_E_INVALID, "vopp_pipe_rates: null output or negative capacity");
  }
  *n_out = 0;
  cudaError_t e = cudaSetDevice(device);
  int sms = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess || sms <= 0) {
    return vopp::set_error(VOPP_E_CUDA, (std::string("vopp_pipe_rates: ") +
                                         cudaGetErrorString(e)).c_str());
  }
  const unsigned grid = (unsigned)(sms * kBlocksPerSm);
  BlockClock *clocks = nullptr;
  uint32_t *sink = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  e = cudaMalloc(&clocks, sizeof(BlockClock) * grid);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(uint32_t) * grid * kThreads);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[0]);
  if (e == cudaSuccess) e = cudaEventCreate(&ev[1]);
  std::vector<BlockClock> h(grid);
  const int n = max_out < OP_COUNT ? max_out : OP_COUNT;
  for (int op = 0; op < n && e == cudaSuccess; ++op) {
    e = launch_any(op, grid, clocks, sink, s);                       // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(ev[0], s);
    if (e == cudaSuccess) e = launch_any(op, grid, clocks, sink, s);
    if (e == cudaSuccess) e = cudaEventRecord(ev[1], s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    if (e == cudaSuccess)
      e = cudaMemcpy(h.data(), clocks, sizeof(BlockClock) * grid, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) break;
    // per SM: operations of its CTAs over the cycles from its first start to its last end
    std::vector<long long> first(sms, 0), last(sms, 0);
    std::vector<int> blocks(sms, 0);
    for (const BlockClock &b : h) {
      if ((int)b.smid >= sms) continue;
      if (blocks[b.smid] == 0 || b.start < first[b.smid]) first[b.smid] = b.start;
      if (blocks[b.smid] == 0 || b.end > last[b.smid]) last[b.smid] = b.end;
      ++blocks[b.smid];
    }
    const double ops_per_block = (double)kThreads * kChains * kIters;
    double rate_sum = 0.0;
    int used = 0;
    for (int m = 0; m < sms; ++m) {
      if (blocks[m] == 0 || last[m] <= first[m]) continue;
      rate_sum += blocks[m] * ops_per_block / (double)(last[m] - first[m]);
      ++used;
    }
    vopp_pipe_rate &r = out[op];
    std::memset(&r, 0, sizeof(r));
    std::strncpy(r.op, kOpNames[op], sizeof(r.op) - 1);
    r.thread_ops_per_clock_per_sm = used ? rate_sum / used : 0.0;
    r.ops_per_second = grid * ops_per_block / (ms * 1e-3);
    r.sms = sms;
    *n_out = op + 1;
  }
  if (ev[0]) cudaEventDestroy(ev[0]);
  if (ev[1]) cudaEventDestroy(ev[1]);
  if (s) cudaStreamDestroy(s);
  if (sink) cudaFree(sink);
  if (clocks) cudaFree(clocks);
  if (e != cudaSuccess)
    return vopp::set_error(VOPP_E_CUDA, (std::string("vopp_pipe_rates: ") +
                                         cudaGetErrorString(e)).c_str());
  return VOPP_OK;
}
