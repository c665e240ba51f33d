// Parameter blocks of the GOM-step kernels (gom.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "isa.h"

namespace gg {

struct GomDonateParams {
  int n, stride, n_fos, n_pop;
  uint8_t* op;            // offspring [n][stride], modified in place
  float* cval;
  const uint8_t* pop_op;  // population (donors) [n_pop][stride]
  const float* pop_cval;
  const int* donor;       // [n]
  const int* subset;      // [n] FOS index per offspring
  const int* fos_off;     // [n_fos + 1]
  const int* fos_nodes;   // template positions of every subset
};

struct GomChangedParams {
  int n, stride, h_max, layout, n_features;
  const uint8_t* op;      // offspring
  const float* cval;
  const int8_t* height;   // nullable
  const uint8_t* bop;     // backup
  const float* bcval;
  uint8_t* changed;       // [n]
};

struct GomAcceptParams {
  int n, stride;
  uint8_t* op;            // offspring, reverted in place
  float* cval;
  uint8_t* bop;           // backup, updated in place
  float* bcval;
  const uint8_t* changed; // nullable: every offspring changed
  const float* f_new;
  float* f_old;           // backup fitness, updated in place
  uint8_t* accepted;      // nullable
};

struct TrialSizeParams {
  int n, stride, h_max, layout, n_features;
  const uint8_t* op;
  const int8_t* height;   // nullable
  int* size;              // [n]
};

const void* trial_size_ptr();
const void* gom_donate_ptr();
const void* gom_changed_ptr();
const void* gom_accept_ptr();

}  // namespace gg
