// Launch accounting and the opt-in kernel probe (process-wide).
//
// Every kernel launch of the library goes through probed(): it counts the
// launch, and when a probe is armed for the launch's (kind, precision) it
// records a CUDA event pair around the launch on the launching stream and
// hands the kernel a device counter that each block which does work (i.e.
// is not gated off) increments once.  The algorithmic bytes of the probed
// launches are then (blocks that ran) x (bytes one block must move).  The
// event pool holds a fixed number of pairs; launches beyond it are counted
// but neither timed nor added to the byte counter.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <vector>

namespace wz {

enum ProbeKind { PK_ZT = 0, PK_XY = 1, PK_CG_P1 = 2, PK_CG_P3 = 3, PK_CG_P5 = 4, PK_RU_P1 = 5, PK_RU_P5 = 6 };

struct Probe {
  int active = 0;
  int kind = -1;
  int real_bytes = 0;  // 4: FP32 kernels, 8: FP64 kernels
  unsigned long long* d_blocks = nullptr;
  std::vector<cudaEvent_t> ev;  // start/stop pairs
  int recorded = 0;
  long launches = 0;
  double bytes_per_block = 0.0;
};

extern Probe g_probe;
extern std::atomic<unsigned long long> g_launches;  // process-wide
extern thread_local unsigned long long tl_launches;  // this host thread

inline void count_launch(unsigned long long n = 1) {
  g_launches += n;
  tl_launches += n;
}

template <class F>
inline cudaError_t probed(int kind, int real_bytes, double bytes_per_block, cudaStream_t st, F launch) {
  count_launch();
  Probe& p = g_probe;
  const bool on = p.active && p.kind == kind && p.real_bytes == real_bytes;
  if (!on) return launch((unsigned long long*)nullptr);
  const int pair = p.recorded;
  const bool rec = 2 * pair + 1 < (int)p.ev.size();
  // only a launch with an event pair adds its bytes: achieved = bytes / time
  // then covers the same launches on both sides of the division
  if (!rec) {
    p.launches += 1;
    return launch((unsigned long long*)nullptr);
  }
  cudaEventRecord(p.ev[2 * pair], st);
  cudaError_t e = launch(p.d_blocks);
  cudaEventRecord(p.ev[2 * pair + 1], st);
  p.recorded += 1;
  p.launches += 1;
  p.bytes_per_block = bytes_per_block;
  return e;
}

}  // namespace wz
