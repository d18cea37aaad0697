// camp_solve_host_static: the host-staged solve for callers that cannot
// allocate device memory.  Its staging buffers and work counter live in one
// file-scope device array of CAMP_STATIC_SCRATCH_BYTES; host code only ever
// passes the array's device address, fetched per device with
// cudaGetSymbolAddress (the array's name is not a device address in host
// code).
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "camp.h"
#include "launch.h"

static __device__ __align__(256) unsigned char camp_static_scratch[CAMP_STATIC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_mu;                    // one call at a time: they share the array
void *g_scratch[kMaxDevices] = {};  // device address of the array, per device

size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }
}  // namespace

extern "C" int camp_solve_host_static(const camp_mech *m, int64_t n_cells, double *state,
                                      const double *env, double dt, double rtol, const double *atol,
                                      int32_t atol_len, int32_t *status, const camp_solve_opts *opts,
                                      void *stream) {
    camp_mech_info inf;
    if (!m || camp_mech_info_get(m, &inf) != CAMP_OK) return camp_record_error(CAMP_E_INVAL, "NULL mechanism");
    if (camp_mech_needs_scratch(m))
        return camp_record_error(CAMP_E_UNSUPPORTED, "a block-arrow (particle-resolved) mechanism needs per-cell scratch; "
                                                     "use camp_solve_host");
    if (n_cells < 0) return camp_record_error(CAMP_E_INVAL, "n_cells < 0");
    if (n_cells == 0) return CAMP_OK;
    if (!state || !env || !atol || !status) return camp_record_error(CAMP_E_INVAL, "NULL array");
    if (atol_len != 1 && atol_len != inf.n_species)
        return camp_record_error(CAMP_E_INVAL, "atol_len must be 1 or n_species");
    int32_t *host_stats = opts ? opts->stats : nullptr;
    double *host_step = opts ? opts->step : nullptr;
    const size_t b_step = host_step ? al256((size_t)n_cells * 8) : 0;
    const size_t b_state = al256((size_t)n_cells * inf.n_species * 8);
    const size_t b_env = al256((size_t)n_cells * inf.n_env * 8);
    const size_t b_status = al256((size_t)n_cells * 4);
    const size_t b_atol = al256((size_t)atol_len * 8);
    const size_t b_stats = host_stats ? al256((size_t)n_cells * 4 * CAMP_NSTATS) : 0;
    const size_t b_ws = al256(camp_workspace_bytes());
    const size_t need = b_state + b_env + b_status + b_atol + b_stats + b_ws + b_step;
    if (need > (size_t)CAMP_STATIC_SCRATCH_BYTES) {
        std::string msg = "chunk needs " + std::to_string(need) + " bytes of staging, more than the " +
                          std::to_string((size_t)CAMP_STATIC_SCRATCH_BYTES) +
                          "-byte static scratch; split it or use camp_solve_host";
        return camp_record_error(CAMP_E_INVAL, msg.c_str());
    }

    std::lock_guard<std::mutex> lk(g_mu);
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
        return camp_record_error(CAMP_E_CUDA, "no usable current device");
    if (!g_scratch[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, camp_static_scratch);
        if (e != cudaSuccess || !p)
            return camp_record_error(CAMP_E_CUDA, (std::string("cudaGetSymbolAddress: ") +
                                                   cudaGetErrorString(e)).c_str());
        g_scratch[dev] = p;
    }
    char *base = (char *)g_scratch[dev];
    double *d_state = (double *)base;
    double *d_env = (double *)(base + b_state);
    int32_t *d_status = (int32_t *)(base + b_state + b_env);
    double *d_atol = (double *)(base + b_state + b_env + b_status);
    int32_t *d_stats = host_stats ? (int32_t *)(base + b_state + b_env + b_status + b_atol) : nullptr;
    void *d_ws = base + b_state + b_env + b_status + b_atol + b_stats;
    double *d_step = host_step ? (double *)(base + b_state + b_env + b_status + b_atol + b_stats + b_ws) : nullptr;

    cudaStream_t s = (cudaStream_t)stream;
    // Once a copy is enqueued, every return waits for the stream first: the
    // lock is released on return, and the next call (perhaps on another
    // stream) must not overwrite the array while this call's work is in
    // flight.
    auto drain = [&](int code, const std::string &msg) {
        cudaStreamSynchronize(s);
        if (code == CAMP_OK) return CAMP_OK;
        return msg.empty() ? code : camp_record_error(code, msg.c_str());
    };
    const size_t n_state = (size_t)n_cells * inf.n_species * 8, n_env = (size_t)n_cells * inf.n_env * 8;
    cudaError_t e = cudaMemcpyAsync(d_state, state, n_state, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_env, env, n_env, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_atol, atol, (size_t)atol_len * 8, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && host_step) e = cudaMemcpyAsync(d_step, host_step, (size_t)n_cells * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return drain(CAMP_E_CUDA, std::string("staging copy: ") + cudaGetErrorString(e));
    camp_solve_opts o;
    camp_solve_opts_default(&o, opts ? opts->variant : CAMP_VARIANT_MIXED);
    if (opts) o = *opts;
    o.stats = d_stats;
    o.step = d_step;
    o.workspace = d_ws;  // the persistent grid's counter: zeroed by camp_solve
    int rc = camp_solve(m, n_cells, d_state, d_env, dt, rtol, d_atol, atol_len, d_status, &o, stream);
    if (rc != CAMP_OK) return drain(rc, "");  // camp_solve recorded the message
    e = cudaMemcpyAsync(state, d_state, n_state, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(status, d_status, (size_t)n_cells * 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && host_stats)
        e = cudaMemcpyAsync(host_stats, d_stats, (size_t)n_cells * 4 * CAMP_NSTATS, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && host_step)
        e = cudaMemcpyAsync(host_step, d_step, (size_t)n_cells * 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return drain(CAMP_E_CUDA, std::string("result copy: ") + cudaGetErrorString(e));
    return CAMP_OK;
}
