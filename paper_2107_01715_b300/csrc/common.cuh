// common.cuh -- shared definitions of the CUDA side of libbcts (not shared with
// the oracle, which restates everything on its own).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/bcts.h"

namespace bcts {

// Sprite-environment geometry (the stand-in for the paper's Atari simulator).
constexpr int kGrid = 21;        // cells per side
constexpr int kHist = 4;         // frames per stack (Sec. 5 frame stacking)
constexpr int kObj = 4;          // agent, reward, two hazards
constexpr int kPix = 84;         // pixels per side, 4x4 pixels per cell
constexpr int kFrameBytes = kHist * kPix * kPix;  // 28,224
constexpr int kStateBytes = 80;
constexpr int kMaxA = 18;
constexpr int kMaxDepth = 6;

static_assert(sizeof(bcts_state) == kStateBytes, "state layout");

// Nature-DQN geometry.
constexpr int kC1 = 32, kC2 = 64, kC3 = 64, kF1 = 512;
constexpr int kK1 = 4 * 8 * 8;    // 256
constexpr int kK2 = 32 * 4 * 4;   // 512
constexpr int kK3 = 64 * 3 * 3;   // 576
constexpr int kKF = 64 * 7 * 7;   // 3136
constexpr int kP1 = 20 * 20, kP2 = 9 * 9, kP3 = 7 * 7;

// Status plumbing: every host helper returns a bcts status and records a message.
struct Status {
  int code = BCTS_OK;
  std::string msg;
};

void set_thread_error(const std::string &msg);
const char *thread_error();

// ---- per-kernel-class timing (CUDA events on the launching stream) ----------
// Kernel classes, same numbering as BCTS_KERN_* in bcts.h.
enum KernelKind {
  K_EXPAND = 0, K_RENDER, K_CONV1, K_CONV2, K_CONV3, K_FC1, K_FC2, K_BACKUP, K_CONV1_PARTIAL, K_CONV1_LEAF,
  K_DNN_MLP, K_DNN_Q, K_COUNT
};

struct Profiler;
// The profiler of the context running on this thread (NULL outside a context).
Profiler *&thread_profiler();
void prof_begin(int kind, cudaStream_t st);
void prof_end(int kind, cudaStream_t st);

struct ProfScope {
  int kind;
  cudaStream_t st;
  ProfScope(int k, cudaStream_t s) : kind(k), st(s) { prof_begin(k, s); }
  ~ProfScope() { prof_end(kind, st); }
};

struct ProfilerGuard {
  Profiler *prev;
  explicit ProfilerGuard(Profiler *p) : prev(thread_profiler()) { thread_profiler() = p; }
  ~ProfilerGuard() { thread_profiler() = prev; }
};

}  // namespace bcts

#define BCTS_CUDA_TRY(call, errstr)                                                           \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess) {                                                                  \
      (errstr) = std::string(#call) + ": " + cudaGetErrorString(e_);                          \
      return BCTS_ECUDA;                                                                      \
    }                                                                                         \
  } while (0)
