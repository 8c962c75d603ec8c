// echo_ctx.h -- the host-side context behind the opaque echo_ctx handle
// (internal; shared by echo_api.cu and echo_batch.cu).
#pragma once

#include <string>
#include <vector>

#include "../../include/echo.h"
#include "echo_device.cuh"

using echo::Arrays;
using echo::Geom;
using echo::Phys;

struct echo_ctx {
    echo_grid grid;
    echo_metric metric;
    echo_eos eos;
    int precision;
    double cfl;
    Geom geo;
    Phys ph;
    size_t ws_need = 0;
    char *ws = nullptr;
    cudaStream_t stream = nullptr;
    bool bound = false;
    bool have_state = false;
    Arrays<double> ad;
    Arrays<float> af;
    size_t nstate = 0;
    long long ntiles = 0;     // tiles of 128 owned cells (c2p, network starts)
    size_t staging_count = 0;
    int nblk_red = 0;
    std::string err;
    int c2p_guess = 0;        // 0 previous-stage Z, 1 c2p-guess network
    bool mlp_loaded = false;
    bool ze_valid = false;    // the per-cell start codes and the list describe the current Newton memory
    int ze_refine = -1;       // the FP32-refinement flag (mode +4) of the gate that made the list; -1 either
    // per-kernel timing (echo_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev;      // pool, pairs (start, end)
    std::vector<int> ev_kind;         // kernel class of each recorded pair
    size_t ev_used = 0;               // pairs in use
};

// Before an inversion with guess mode `mode` on stream s: a network mode
// whose start codes are stale (plain-mode inversions ran since they were
// written) resets them to "previous Z exact"; a plain mode marks them stale
// (internal).
extern "C" __attribute__((visibility("hidden"))) int echo_internal_prepare_start(echo_ctx *c, int mode, cudaStream_t s);

// One step of c enqueued on stream s instead of its own (internal).
extern "C" __attribute__((visibility("hidden"))) int echo_internal_enqueue_step(echo_ctx *c, double dt, cudaStream_t s);
