// Host-side state of one volume (the opaque rf_volume of refusion.h).
#pragma once

#include <string>
#include <vector>

#include "rf_internal.cuh"

struct rf_graph_entry {
  int H, W;
  double fx, fy, cx, cy;
  int first;      // first frame: integrate only
  int profiling;  // graph holds the profiling event records
  cudaGraphExec_t exec;
};

struct rf_volume {
  rf_params p;
  rf::DevParams dp;
  rf::DevVol dv;
  int64_t n_buckets = 0, max_blocks = 0;
  int max_w = 0, max_h = 0;
  int device = 0, sm_count = 0;
  size_t device_bytes = 0;

  // model
  unsigned long long* d_hash = nullptr;
  uint2* d_vox = nullptr;
  uint8_t* d_W = nullptr;
  int4* d_coords = nullptr;
  int4* d_nbr = nullptr;
  int* d_nblocks = nullptr;
  unsigned* d_status = nullptr;

  // registration scratch
  // 2 x 29 x max_slots tagged partial sums of the registration (tag << 32 |
  // float bits).  Mesh extraction and virtual-depth filling reuse word 0 as a
  // counter between registrations: a count below 2^32 in it, or in its low
  // half, leaves a tag no later registration waits for.
  unsigned long long* d_partials = nullptr;
  int max_slots = 0;
  unsigned* d_regtags = nullptr;  // registration tag base and leaving count
  int reg_grid = 0;

  // mask scratch
  uint8_t* d_seeds = nullptr;
  uint8_t* d_md = nullptr;     // M_D during the flood fill
  unsigned* d_ff = nullptr;    // barrier words + per-sweep change flags
  int ff_grid = 0;

  // integration scratch
  rf::IntegState* d_integ = nullptr;
  int* d_tilemax = nullptr;
  uint16_t* d_dmask = nullptr;  // per pixel: raw depth if valid and not masked, else 0
  int4* d_cand = nullptr;

  // whole-frame staging (graph-replayed pipeline reads only these)
  uint16_t* d_depth = nullptr;
  uint8_t* d_rgb = nullptr;
  uint8_t* d_mask = nullptr;
  double* d_T = nullptr;        // [3][16]: T_in, T_first, T_second
  rf_track_info* d_info = nullptr;

  unsigned* d_guard = nullptr;  // FP64 re-evaluated seed count of the last mask
  unsigned long long* d_pxcache = nullptr;  // per pixel: block key << 22 | pool of its last sample

  // profiling: events recorded around the stages of the whole-frame calls
  bool profiling = false;
  cudaEvent_t ev[rf::EV_COUNT] = {};

  // bounded waits of the grid barriers (rf_set_wait_limits)
  long long wait_spins = rf::kDefaultSpinLimit;
  unsigned wait_extra = 0;

  // launch shapes (grid = SMs x CTAs per SM), set by rf_set_launch_config
  rf_launch_config launch = {16, 8, 2, 8, 16};

  std::vector<rf_graph_entry> graphs;
  bool use_graphs = true;
  int64_t frames = 0;
  bool has_model = false;  // false: the next frame is integrated at its T_init without tracking
  std::string last_error;
};
