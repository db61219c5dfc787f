// resident_kernels.cuh — the batched persistent kernel kept resident for a
// server: its producer warps take tiles from a ring that the host fills while
// the kernel runs, so a request reaches the GPU without a kernel launch.
//
// Host and device share, in page-locked mapped host memory:
//   - a request table (ResidentReq per slot: the nest descriptor, the number
//     of tiles of the request and its sequence number in the slot),
//   - a tile ring (BatchTile, nest = request slot),
//   - a control block per kernel instance (tiles published, stop flag),
//   - a completion word per slot (the sequence number of the slot's last
//     finished request).
// The host writes a request's descriptor and tiles, then publishes them by
// raising the instance's tail with a release store.  Producers claim tile
// indices from a device counter; the one holding the first unpublished index
// (the head waiter) polls the host's tail and mirrors it into device memory,
// where the other waiters read it (eight copies on separate lines, so that
// hundreds of idle producers do not load one L2 slice).  Every tile runs the
// batched executor's code unchanged, so results are bit-identical to
// hp_nest_run.  After a tile the consumer warps meet at a barrier, one thread
// fences and counts the tile against its request; the CTA that finishes the
// last tile fences at system scope and writes the request's sequence number to
// the completion word, which the host polls.
//
// Every wait is bounded.  A producer waits for one tile at most cap_ns
// (global timer), then records status 4, mirrors a stop to the other waiters
// and leaves; the host sets the stop flag long before that (an instance lives
// for one epoch of host time, or until the server has been idle for 2 ms) and
// launches the next instance.  The consumer wait for the next queued tile is
// bounded by cap_ns plus one second.
#pragma once

#include "batch_kernels.cuh"

namespace hp {

#ifndef HP_RESIDENT_NAP_NS
#define HP_RESIDENT_NAP_NS 256u                  // a waiter's pause between reads of its mirror copy
#endif
constexpr int kResidentMirrors = 8;              // copies of the mirrored tail / stop words
constexpr int kResidentLineWords = 16;           // one 128-byte line per copy
constexpr int kResidentDevWords = kResidentLineWords * (1 + kResidentMirrors);
constexpr int32_t kErrResidentCap = 4;           // a producer's wait for one tile reached cap_ns

// per kernel instance, in mapped host memory (written by the host)
struct ResidentCtl {
  unsigned long long tail;   // tiles published to the instance
  unsigned long long stop;   // nonzero: leave once every published tile is taken
};

// per request slot, in mapped host memory (written by the host); whole
// 128-byte lines, so that no two slots share a line
struct alignas(128) ResidentReq {
  BatchNest bn;
  int32_t n_tiles;
  uint32_t seq;
};
static_assert(sizeof(BatchNest) % 8 == 0 && sizeof(ResidentReq) % 128 == 0, "8-byte copies of whole lines");
static_assert(sizeof(BatchNest) / 8 >= 32 && sizeof(BatchNest) / 8 + 1 <= 64,
              "a warp copies a descriptor and its (n_tiles, seq) word in two loads per lane");

__device__ __forceinline__ unsigned long long ld_acquire_sys(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.sys.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_gpu(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];\n" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_sys(int32_t* p, int32_t v) {
  asm volatile("st.relaxed.sys.global.s32 [%0], %1;\n" ::"l"(p), "r"(v) : "memory");
}
// strong (volatile) loads of host-written words: a slot or ring line the GPU
// read before may have been rewritten by the host since, so no cached copy
// of it may serve these reads
__device__ __forceinline__ int2 ld_volatile2(const int2* p) {
  int2 v;
  asm volatile("ld.volatile.global.v2.s32 {%0, %1}, [%2];\n" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int4 ld_volatile4(const int4* p) {
  int4 v;
  asm volatile("ld.volatile.global.v4.s32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}

struct ResidentSource {
  static constexpr bool kResident = true;
  const ResidentReq* reqs;       // mapped host memory, one per slot
  const BatchTile* ring;         // mapped host memory, ring_mask + 1 entries
  unsigned long long ring_mask;
  unsigned long long base;       // ring index of the instance's first tile
  const ResidentCtl* ctl;        // mapped host memory
  unsigned long long* dev;       // device: [0] tiles claimed; line c+1: [0] tail seen, [1] stop seen
  int32_t* counts;               // device: tiles finished per slot (0 between requests)
  uint32_t* done;                // mapped host memory: per slot, seq of its last finished request
  int32_t* status;               // mapped host memory: 0, kErrStageWait or kErrResidentCap
  unsigned long long cap_ns;     // longest wait for one tile

  // publish a value to every mirror copy (word w of each line): one fence
  // orders what this thread observed before it, then relaxed maxima
  __device__ __forceinline__ void mirror_all(int w, unsigned long long v) const {
    __threadfence();
#pragma unroll
    for (int c = 0; c < kResidentMirrors; ++c) atomicMax(dev + kResidentLineWords * (1 + c) + w, v);
  }
  // lane 0: the next published tile, or -1 once the instance stops (or its cap passes)
  __device__ int64_t claim() const {
    const unsigned long long k = atomicAdd(dev, 1ull);
    unsigned long long* mirror = dev + kResidentLineWords * (1 + (blockIdx.x % kResidentMirrors));
    const unsigned long long t_end = global_ns() + cap_ns;
    for (uint32_t i = 1;; ++i) {
      const unsigned long long seen = ld_acquire_gpu(mirror);
      if (k < seen) return static_cast<int64_t>(k);
      if (k == seen) {
        // the head waiter polls the host's tail; every 8th poll it reads the
        // stop flag first and the tail after it, so that a stop seen comes
        // with the final tail
        const bool check_stop = (i & 7u) == 0;
        const unsigned long long st = check_stop ? ld_acquire_sys(&ctl->stop) : 0ull;
        const unsigned long long tl = ld_acquire_sys(&ctl->tail);
        if (tl > seen) mirror_all(0, tl);
        if (k < tl) return static_cast<int64_t>(k);
        if (st) {
          mirror_all(1, 1ull);
          return -1;
        }
      } else if (ld_acquire_gpu(mirror + 1)) {
        // stop was mirrored by a head waiter after the final tail
        if (k < ld_acquire_gpu(mirror)) return static_cast<int64_t>(k);
        return -1;
      }
      if ((i & 15u) == 0 && global_ns() > t_end) {
        st_relaxed_sys(status, kErrResidentCap);
        mirror_all(1, 1ull);
        return -1;
      }
      if (k != seen) __nanosleep(HP_RESIDENT_NAP_NS);
    }
  }
  __device__ __forceinline__ BatchTile tile(int64_t k) const {
    const int4 v = ld_volatile4(reinterpret_cast<const int4*>(ring + ((base + static_cast<unsigned long long>(k)) & ring_mask)));
    BatchTile t;
    t.nest = v.x;
    t.count = v.y;
    t.item0 = static_cast<int64_t>((static_cast<uint64_t>(static_cast<uint32_t>(v.w)) << 32) |
                                   static_cast<uint32_t>(v.z));
    return t;
  }
  // the slot's descriptor and (n_tiles, seq): 45 words of 8 bytes, every load
  // issued before the first store, so the host link is crossed once
  __device__ __forceinline__ void desc(int lane, const BatchTile& t, BatchQueued& e) const {
    constexpr int kWords = static_cast<int>(sizeof(BatchNest) / 8);
    const int2* src = reinterpret_cast<const int2*>(reqs + t.nest);
    int2* dst = reinterpret_cast<int2*>(&e.bn);
    const int2 v0 = ld_volatile2(src + lane);
    const bool two = lane + 32 <= kWords;   // word kWords is (n_tiles, seq)
    int2 v1 = make_int2(0, 0);
    if (two) v1 = ld_volatile2(src + lane + 32);
    dst[lane] = v0;
    if (two) {
      if (lane + 32 < kWords) {
        dst[lane + 32] = v1;
      } else {
        e.req_tiles = v1.x;
        e.req_seq = static_cast<uint32_t>(v1.y);
      }
    }
  }
  __device__ __forceinline__ void report(int32_t code) const { st_relaxed_sys(status, code); }
  __device__ __forceinline__ unsigned long long idle_limit_ns() const { return cap_ns + kBatchWaitNs; }
  // all consumer threads, after a tile: count it against its request; the
  // last tile of a request publishes the request's completion to the host
  // (the barrier orders every consumer's writes before thread 0's fence, and
  // fences are cumulative: one fence per tile publishes the whole CTA's)
  __device__ __forceinline__ void tile_done(const BatchQueued& e, uint32_t abort_at) const {
    const bool aborted = consumer_sync_or(ld_abort(abort_at));
    if (!aborted && threadIdx.x == 0) {
      const int32_t slot = e.t.nest;
      __threadfence();   // the CTA's outputs, partials and tickets are visible GPU-wide
      if (atomicAdd(&counts[slot], 1) == e.req_tiles - 1) {
        counts[slot] = 0;   // ready for the slot's next request
        __threadfence_system();
        st_relaxed_sys(reinterpret_cast<int32_t*>(done + slot), static_cast<int32_t>(e.req_seq));
      }
    }
  }
};

template <class Op>
__global__ void __launch_bounds__(kBatchAllThreads, HP_BATCH_MIN_BLOCKS) resident_kernel(ResidentSource src) {
  batch_cta<Op>(src);
}

template <class Op>
inline cudaError_t launch_resident_op(const ResidentSource& src, int grid, cudaStream_t st) {
  static const cudaError_t attr =
      cudaFuncSetAttribute(resident_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
  if (attr != cudaSuccess) return attr;
  resident_kernel<Op><<<grid, kBatchAllThreads, kRingBytes, st>>>(src);
  return cudaPeekAtLastError();
}

template <class Op>
inline int resident_blocks_per_sm() {
  static const cudaError_t attr =
      cudaFuncSetAttribute(resident_kernel<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, kRingBytes);
  if (attr != cudaSuccess) return 1;
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, resident_kernel<Op>, kBatchAllThreads, kRingBytes);
  return n < 1 ? 1 : n;
}

// the arithmetics a resident server runs (batch_combo numbering): FP32 sum,
// compensated sum, max, min and int32 sum, max, min
inline bool resident_combo_ok(int combo) { return combo >= 0 && combo <= 6; }
cudaError_t launch_resident_combo(int combo, const ResidentSource& src, int grid, cudaStream_t st);  // resident_*.cu
int resident_combo_blocks_per_sm(int combo);

}  // namespace hp
