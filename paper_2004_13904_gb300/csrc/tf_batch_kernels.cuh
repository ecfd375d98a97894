// Persistent batch kernel: the generic engine's product stages of many problems (App. A
// per problem) in one launch.  Resident CTAs claim work items (tiles of columns) in
// increasing order from a device counter; an item of a stage that needs an earlier stage
// of the same problem and column waits, thread 0 spinning on that stage's per-column
// counter.  Every wait is bounded: past the launch's budget the waiting CTA records
// TF_ETIMEOUT in the status word and returns, and the other CTAs return at their next
// check, so the host reads an error status instead of the GPU hanging.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>

#include "tf_check.cuh"
#include "tf_generic.cuh"
#include "tf_internal.h"

namespace tfk {

namespace {

using namespace gen;

constexpr int kStatusTimeout = 6;  // TF_ETIMEOUT

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int load_volatile(const int* p) { return *(volatile const int*)p; }

// Thread 0 waits until *p >= target (then acquires: the producer's writes are visible),
// the batch's status is set by another CTA, or the deadline passes (then it records
// TF_ETIMEOUT).  A spin count cap backs the clock check.  Returns true on success.
__device__ bool bounded_wait(const int* p, int target, unsigned long long deadline, int* status) {
  for (long long spin = 0;; ++spin) {
    if (load_volatile(p) >= target) {
      __threadfence();
      return true;
    }
    if (load_volatile(status) != 0) return false;
    if (global_ns() > deadline || spin > (1ll << 26)) {
      atomicCAS(status, 0, kStatusTimeout);
      return false;
    }
    __nanosleep(128);
  }
}

// Compiled for at least three resident CTAs per SM (at most 85 registers a thread): on the
// 64 problems of the fifth configuration (32 columns, FP32, 8 x 8 tiles) 16.7 -> 12.2 ms
// per pass against the compiler's default budget.
template <typename T, int TB, int TK>
__global__ void __launch_bounds__(kThreads, 3) k_batch(const BatchCtl c) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(16) BatchArgs<T> s_args;
  __shared__ long long s_item;
  __shared__ int s_seg, s_go;
  __shared__ unsigned long long s_deadline;
  if (threadIdx.x == 0) {
    s_deadline = global_ns() + c.budget_ns;
    s_go = c.gate ? bounded_wait(c.gate, 1, s_deadline, c.status) : 1;
  }
  __syncthreads();
  if (!s_go) return;
  unsigned long long next = 0, end = 0;  // thread 0's claimed items [next, end)
  for (;;) {
    __syncthreads();  // the previous item's shared-memory use is over
    if (threadIdx.x == 0) {
      int go = 0;
      if (next >= end) {
        next = atomicAdd(c.work, (unsigned long long)c.claim);
        end = next + (unsigned long long)c.claim;
      }
      if (next < (unsigned long long)c.total && load_volatile(c.status) == 0) {
        int lo = 0, hi = c.nseg - 1;  // last segment with first <= next
        while (lo < hi) {
          const int mid = (lo + hi + 1) / 2;
          if ((unsigned long long)c.seg[mid].first <= next) lo = mid; else hi = mid - 1;
        }
        const BatchSeg sg = c.seg[lo];
        const int col = (int)((long long)(next - sg.first) / sg.tiles);
        go = sg.wait < 0 ? 1
                         : (bounded_wait(c.counters + sg.wait + col, sg.wait_target, s_deadline,
                                         c.status) ? 1 : 0);
        s_seg = lo;
        s_item = (long long)next;
      }
      ++next;
      s_go = go;
    }
    __syncthreads();
    if (!s_go) return;
    const BatchSeg sg = c.seg[s_seg];
    {
      const int* src = reinterpret_cast<const int*>(static_cast<const BatchArgs<T>*>(c.args) + sg.args);
      int* dst = reinterpret_cast<int*>(&s_args);
      for (int i = threadIdx.x; i < (int)(sizeof(BatchArgs<T>) / sizeof(int)); i += blockDim.x)
        dst[i] = src[i];
    }
    __syncthreads();
    const long long local = s_item - sg.first;
    const int col = (int)(local / sg.tiles), tile = (int)(local % sg.tiles);
    switch (sg.kind) {
      case 0: rows_r2c_body<T, TB>(s_args.r2c, tile, col, smem_raw); break;
      case 1: cols_fwd_body<T, TK>(s_args.fwd, tile, col, smem_raw); break;
      case 2: rows_c2r_body<T, TB>(s_args.c2r, tile, col, smem_raw); break;
      default: cols_adj_body<T, TK>(s_args.adj, tile, col, smem_raw); break;
    }
    __threadfence();   // this thread's stores of the tile, device-wide
    __syncthreads();   // all threads' stores issued and fenced
    if (threadIdx.x == 0) atomicAdd(c.counters + sg.count + col, 1);
  }
}

template <auto Kernel>
cudaError_t prep_smem(size_t smem) {
  static std::atomic<size_t> granted[64];
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64)
    return cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  size_t have = granted[dev].load(std::memory_order_relaxed);
  if (smem <= have) return cudaSuccess;
  e = cudaFuncSetAttribute(Kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    while (have < smem && !granted[dev].compare_exchange_weak(have, smem)) {}
  return e;
}

template <typename T, int TB, int TK>
cudaError_t batch_tiles(const BatchCtl& c, size_t smem, cudaStream_t s, int* grid) {
  constexpr auto K = k_batch<T, TB, TK>;
  cudaError_t e = prep_smem<K>(smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0, dev = 0, sms = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, K, kThreads, smem)) != cudaSuccess) return e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const long long claims = (c.total + c.claim - 1) / c.claim;
  const int g = (int)std::max<long long>(1, std::min<long long>((long long)per_sm * sms, claims));
  K<<<g, kThreads, smem, s>>>(c);
  if (grid) *grid = g;
  return cudaGetLastError();
}

}  // namespace

// The dtype's launcher over its compiled tile pairs (rows tile TB, column tile TK); each
// instantiating translation unit lists its pairs, so the dtypes compile in parallel.
#define TF_BATCH_CASE(TB, TK) \
  case TB * 100 + TK: return batch_tiles<T, TB, TK>(c, smem, s, grid);

}  // namespace tfk
