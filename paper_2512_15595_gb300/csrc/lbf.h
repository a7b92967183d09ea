// Shared definitions of the learned prefilter's integer model: layer sizes,
// the device image of an exported model and the model handle.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "bloomgb.h"

namespace lbf {

constexpr int kIn = 64, kH1 = 128, kH2 = 64;

// Device image: W1T int8 [128][64] (output-major), W2T int8 [64][128], W3
// int8 [64], b1 int32 [128], b2 int32 [64], b3, sh1, sh2 (int32).
constexpr int kImgW1 = 0, kImgW2 = kImgW1 + kH1 * kIn, kImgW3 = kImgW2 + kH2 * kH1, kImgB1 = kImgW3 + kH2,
              kImgB2 = kImgB1 + 4 * kH1, kImgB3 = kImgB2 + 4 * kH2, kImgSh = kImgB3 + 4, kImgBytes = kImgSh + 8;

void image_of(const bf_mlp_int8* m, std::vector<unsigned char>& img);

// Tensor-core form of a model (see lbf_tc.cu): the operand image copied to
// shared memory (weights, bit table), the per-unit requantization constants,
// W3q and the score offset.
struct TcModel {
  std::vector<uint8_t> image;
  long long s3;
  float c1[128];
  float c2[64];
  float w3[64];
};

// A backup filter the tensor-core kernel can probe itself (256-bit blocks,
// S = 32, K = 8, sectorized).
struct TcBackup {
  const uint32_t* words;
  uint64_t num_blocks;
  uint64_t seed;
};

bool tc_eligible(const bf_mlp_int8* m);
bool tc_prepare(const bf_mlp_int8* m, TcModel* out);
uint32_t tc_image_bytes();
// modes: 0 scores to out32, 1 out8[i] = 1 where score >= tau, 4 keys scoring
// below tau appended to out_keys (number in *count), 5 out8[i] = score >= tau
// or `backup` contains key i
cudaError_t tc_run(const uint8_t* d_image, const TcModel& tm, const uint64_t* d_keys, uint64_t n, int mode, int tau,
                   int32_t* out32, uint8_t* out8, unsigned long long* count, uint64_t* out_keys, unsigned int* err,
                   cudaStream_t st, const TcBackup* backup = nullptr);

}  // namespace lbf

struct bf_mlp_model {
  static constexpr int kDepth = 3;  // host pipeline: chunks in flight
  unsigned char* d_img = nullptr;  // CUDA-core image
  uint8_t* d_tc = nullptr;         // tensor-core operand image (null when not eligible)
  unsigned int* d_err = nullptr;   // device error word (bounded waits that ran out)
  lbf::TcModel tc;
  int engine = BF_MLP_ENGINE_AUTO;
  int device = 0;
  // host pipeline (created on first use): staging slots of chunk keys + results
  void* staging = nullptr;
  uint64_t chunk = 0;
  cudaStream_t pipe[kDepth] = {};
  cudaEvent_t ev_done[kDepth] = {};
  cudaEvent_t ev_start = nullptr;
};
