// C ABI of libcamp.so (declared in include/camp.h): argument checking,
// mechanism handles, launch configuration.  No arithmetic of the method lives
// here; every step of the solve runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <stdexcept>
#include <string>

#include "camp.h"
#include "kernels.cuh"
#include "launch.h"
#include "mech.hpp"

struct camp_mech {
    camp::HostMech h;
    DevMech dm;
    void *dev_tables = nullptr;
    int device = 0;
    int sm_count = 0;
    unsigned long long *own_ws = nullptr;
    std::mutex mu;           // guards own_ws creation
    std::mutex stage_mu;     // serialises camp_solve_host's staging buffers
    void *stage = nullptr;
    size_t stage_bytes = 0;
    bool on_device = false;
    int occ[2][9] = {};                 // blocks per SM by variant and cells per block (0 = unknown)
    int tuned_cpb[2] = {0, 0};          // per variant, 0 = untuned
    int tuned_persistent[2] = {-1, -1}; // per variant, -1 = untuned
    // the full mechanism's sizes (h holds the one-particle template when
    // the block-arrow form is used)
    int n = 0, n_env = 0;
    // block-arrow form of a particle-resolved mechanism (arrow.h)
    bool arrow = false;
    camp::ArrowHost ah;
    ArrowDev ad{};
    void *arrow_tables = nullptr;
    int arrow_clusters[2][5] = {};      // co-resident clusters per LU precision and cluster size (0 = unknown)
    // the mechanism text (to rebuild the per-lane tables for another lane
    // count) and the device tables a rebuild replaced: they stay allocated
    // until the mechanism is freed, so that launches already queued or
    // captured in a graph keep valid tables
    std::string json;
    std::vector<void *> old_tables;
};

// CTAs per cluster of the block-arrow solve (default; camp_solve_opts.
// cells_per_block picks 1, 2, 4, 8 or 16 for this form)
static const int kArrowCluster = 8;

// true when camp_solve needs device scratch beyond its arguments and the
// work counter (the block-arrow form's per-cell rows)
bool camp_mech_needs_scratch(const camp_mech *m) { return m && m->arrow; }

namespace {
thread_local std::string g_err;

int fail(int code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(x)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (x);                                                         \
        if (e_ != cudaSuccess)                                                        \
            return fail(CAMP_E_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// dynamic shared memory one block may use (227 KB less room for a block
// group's static reduction scratch)
const int kMaxSmem = 227 * 1024 - 256;

int check_device(const camp_mech *m) {
    if (!m->on_device) return fail(CAMP_E_INVAL, "mechanism was compiled without device tables");
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(CAMP_E_CUDA, "cudaGetDevice failed");
    if (dev != m->device)
        return fail(CAMP_E_INVAL, "current device differs from the mechanism's device");
    return CAMP_OK;
}

template <int G, int NPL, bool W = false>
cudaError_t forcing_npl(const DevMech &m, long long n_cells, const double *state, const double *env,
                        double *f, cudaStream_t s) {
    auto kern = campdev::k_forcing<G, NPL, double, W>;
    int smem = camp_cell_smem_bytes(m, 8);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)n_cells, G, smem, s>>>(m, n_cells, state, env, f);
    return cudaGetLastError();
}
}  // namespace

int camp_record_error(int code, const char *msg) { return fail(code, msg); }

int camp_pick_shape(int n, int lanes) {
    if (n < 1 || n > 2048 || n > 8 * lanes) return -1;
    if (lanes == 32) {
        const int need = (n + 31) / 32;
        const int avail[] = {1, 2, 3, 4, 6, 8};
        for (int a : avail)
            if (a >= need) return a;
    }
    if (lanes == 64 && n <= 256) return CAMP_SHAPE_64X4;
    // blocks of 64, 128, 256 threads with 8 slots a lane
    if (lanes == 64 || lanes == 128 || lanes == 256) return CAMP_SHAPE_BLOCK + lanes / 32;
    return -1;
}

int camp_cell_smem_bytes(const DevMech &m, int lu_elem) {
    return campdev::cell_smem(m.n, m.R, m.n_rev, m.nlu, lu_elem, m.n_part, m.n_pw, m.n_pw64).bytes;
}

cudaError_t camp_launch_rates(const DevMech &m, long long n_cells, const double *env, double *kf,
                              double *kr, cudaStream_t s) {
    const int per = 4;
    campdev::k_rates<32><<<(unsigned)((n_cells + per - 1) / per), 32 * per, 0, s>>>(m, n_cells, env, kf, kr);
    return cudaGetLastError();
}

cudaError_t camp_launch_forcing(const DevMech &m, long long n_cells, const double *state,
                                const double *env, double *f, cudaStream_t s) {
    if (m.n_wsec > 0) {  // the water build: 8-slot shapes only
        switch (camp_pick_shape(m.n, m.lanes) < CAMP_SHAPE_BLOCK ? 8 : camp_pick_shape(m.n, m.lanes)) {
        case 8: return forcing_npl<32, 8, true>(m, n_cells, state, env, f, s);
        case CAMP_SHAPE_64X4: return forcing_npl<64, 4, true>(m, n_cells, state, env, f, s);
        case CAMP_SHAPE_BLOCK + 2: return forcing_npl<64, 8, true>(m, n_cells, state, env, f, s);
        case CAMP_SHAPE_BLOCK + 4: return forcing_npl<128, 8, true>(m, n_cells, state, env, f, s);
        case CAMP_SHAPE_BLOCK + 8: return forcing_npl<256, 8, true>(m, n_cells, state, env, f, s);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (camp_pick_shape(m.n, m.lanes)) {
    case 1: return forcing_npl<32, 1>(m, n_cells, state, env, f, s);
    case 2: return forcing_npl<32, 2>(m, n_cells, state, env, f, s);
    case 3: return forcing_npl<32, 3>(m, n_cells, state, env, f, s);
    case 4: return forcing_npl<32, 4>(m, n_cells, state, env, f, s);
    case 6: return forcing_npl<32, 6>(m, n_cells, state, env, f, s);
    case 8: return forcing_npl<32, 8>(m, n_cells, state, env, f, s);
    case CAMP_SHAPE_64X4: return forcing_npl<64, 4>(m, n_cells, state, env, f, s);
    case CAMP_SHAPE_BLOCK + 2: return forcing_npl<64, 8>(m, n_cells, state, env, f, s);
    case CAMP_SHAPE_BLOCK + 4: return forcing_npl<128, 8>(m, n_cells, state, env, f, s);
    case CAMP_SHAPE_BLOCK + 8: return forcing_npl<256, 8>(m, n_cells, state, env, f, s);
    default: return cudaErrorInvalidValue;
    }
}

extern "C" {

const char *camp_last_error(void) { return g_err.c_str(); }

static int mech_build(const char *json, size_t len, camp_mech **out, char *err, size_t errlen,
                      bool upload) {
    auto report = [&](int code, const std::string &msg) {
        if (err && errlen) {
            size_t k = std::min(errlen - 1, msg.size());
            std::memcpy(err, msg.data(), k);
            err[k] = 0;
        }
        return fail(code, msg);
    };
    if (!out) return report(CAMP_E_INVAL, "out is NULL");
    *out = nullptr;
    if (!json) return report(CAMP_E_INVAL, "json is NULL");
    camp_mech *m = new camp_mech();
    try {
        // a particle-resolved mechanism takes the block-arrow form when it
        // asks for it or is too large for one block's shared memory
        const camp::AerosolShape sh = camp::aerosol_shape(json, len);
        if (sh.particles && sh.instances > 0) {
            camp::HostMech t = camp::compile_mechanism(json, len, 1);
            const long long n_full = t.n_gas + (long long)sh.instances * (t.n - t.n_gas);
            if (sh.block_arrow || n_full > 2048) {
                if (sh.water) throw std::runtime_error("the block-arrow form takes no water parameter");
                m->ah = camp::build_arrow(t, sh.instances);
                m->h = std::move(t);
                m->arrow = true;
            }
        }
        if (!m->arrow) {
            m->h = camp::compile_mechanism(json, len);
            m->json.assign(json, len);
        }
    } catch (const std::exception &e) {
        delete m;
        return report(CAMP_E_PARSE, e.what());
    }
    if (m->arrow) {
        m->n = m->ah.n_g + m->ah.P * m->ah.n_phi;
        m->n_env = m->ah.n_env;
    } else {
        m->n = m->h.n;
        m->n_env = m->h.n_env;
    }
    if (camp_pick_shape(m->h.n, m->h.lanes) < 0) {
        delete m;
        return report(CAMP_E_UNSUPPORTED, "more than 2048 species");
    }
    DevMech probe{};
    std::vector<unsigned char> img = camp::pack_tables(m->h, probe, nullptr);
    if (camp_cell_smem_bytes(probe, 4) > kMaxSmem) {
        delete m;
        return report(CAMP_E_UNSUPPORTED, "per-cell working set exceeds shared memory");
    }
    if (!upload) {
        m->dm = probe;
        *out = m;
        g_err.clear();
        return CAMP_OK;
    }
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, m->device);
    if (e == cudaSuccess) e = cudaMalloc(&m->dev_tables, img.size());
    if (e == cudaSuccess) {
        img = camp::pack_tables(m->h, m->dm, (const unsigned char *)m->dev_tables);
        e = cudaMemcpy(m->dev_tables, img.data(), img.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && m->arrow) {
        ArrowDev probe_a{};
        std::vector<unsigned char> ai = camp::pack_arrow(m->ah, probe_a, nullptr);
        e = cudaMalloc(&m->arrow_tables, ai.size());
        if (e == cudaSuccess) {
            ai = camp::pack_arrow(m->ah, m->ad, (const unsigned char *)m->arrow_tables);
            e = cudaMemcpy(m->arrow_tables, ai.data(), ai.size(), cudaMemcpyHostToDevice);
        }
    }
    if (e != cudaSuccess) {
        if (m->dev_tables) cudaFree(m->dev_tables);
        if (m->arrow_tables) cudaFree(m->arrow_tables);
        delete m;
        return report(e == cudaErrorMemoryAllocation ? CAMP_E_NOMEM : CAMP_E_CUDA,
                      std::string("loading tables: ") + cudaGetErrorString(e));
    }
    m->on_device = true;
    *out = m;
    g_err.clear();
    return CAMP_OK;
}

// Rebuild the mechanism's per-lane tables for `lanes` lanes a cell (the
// integer structure does not change) and make them current; the replaced
// device tables are kept (camp_mech.old_tables).  Synchronous.
static int mech_relane(camp_mech *m, int lanes) {
    if (m->h.lanes == lanes) return CAMP_OK;
    if (m->arrow || m->json.empty()) return fail(CAMP_E_UNSUPPORTED, "no per-lane tables to rebuild");
    camp::HostMech h2;
    try {
        h2 = camp::compile_mechanism(m->json.data(), m->json.size(), -1, lanes);
    } catch (const std::exception &e) {
        return fail(CAMP_E_PARSE, e.what());
    }
    if (camp_pick_shape(h2.n, h2.lanes) < 0) return fail(CAMP_E_UNSUPPORTED, "no cell shape for this lane count");
    DevMech probe{};
    std::vector<unsigned char> img = camp::pack_tables(h2, probe, nullptr);
    if (camp_cell_smem_bytes(probe, 4) > kMaxSmem)
        return fail(CAMP_E_UNSUPPORTED, "per-cell working set exceeds shared memory");
    void *tables = nullptr;
    CUDA_TRY(cudaMalloc(&tables, img.size()));
    DevMech dm2{};
    img = camp::pack_tables(h2, dm2, (const unsigned char *)tables);
    const cudaError_t e = cudaMemcpy(tables, img.data(), img.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(tables);
        return fail(CAMP_E_CUDA, std::string("loading tables: ") + cudaGetErrorString(e));
    }
    m->old_tables.push_back(m->dev_tables);
    m->dev_tables = tables;
    m->h = std::move(h2);
    m->dm = dm2;
    std::memset(m->occ, 0, sizeof m->occ);
    return CAMP_OK;
}

int camp_mech_set_lanes(camp_mech *m, int32_t lanes) {
    if (!m) return fail(CAMP_E_INVAL, "NULL mechanism");
    if (lanes != 32 && lanes != 64 && lanes != 128 && lanes != 256)
        return fail(CAMP_E_INVAL, "lanes per cell must be 32, 64, 128 or 256");
    if (m->arrow) return fail(CAMP_E_UNSUPPORTED, "the block-arrow form has no per-lane tables");
    if (m->h.n > 8 * lanes) return fail(CAMP_E_INVAL, "more than 8 species a lane");
    if (!m->on_device) return fail(CAMP_E_INVAL, "mechanism compiled without a device");
    if (int rc = check_device(m)) return rc;
    return mech_relane(m, lanes);
}

int camp_mech_load(const char *json, size_t len, camp_mech **out, char *err, size_t errlen) {
    return mech_build(json, len, out, err, errlen, true);
}

int camp_mech_compile(const char *json, size_t len, camp_mech **out, char *err, size_t errlen) {
    return mech_build(json, len, out, err, errlen, false);
}

void camp_mech_free(camp_mech *m) {
    if (!m) return;
    if (!m->on_device) {
        delete m;
        return;
    }
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(m->device);
    if (m->dev_tables) cudaFree(m->dev_tables);
    for (void *t : m->old_tables) cudaFree(t);
    if (m->arrow_tables) cudaFree(m->arrow_tables);
    if (m->own_ws) cudaFree(m->own_ws);
    if (m->stage) cudaFree(m->stage);
    if (prev >= 0) cudaSetDevice(prev);
    delete m;
}

int camp_mech_info_get(const camp_mech *m, camp_mech_info *o) {
    if (!m || !o) return fail(CAMP_E_INVAL, "NULL argument");
    const camp::HostMech &h = m->h;
    o->n_species = h.n;
    o->n_rxn = (int32_t)h.procs.size();
    o->n_env = h.n_env;
    o->n_sections = h.n_sections;
    o->nnz_jac = (int32_t)h.colidx.size();
    o->nnz_lu = (int32_t)h.lu_colidx.size();
    o->rxn_map_len = (int32_t)h.rxn_map.size();
    o->dense_block = h.D;
    o->lu_storage = h.nlu;
    o->smem_per_cell_mixed = camp_cell_smem_bytes(m->dm, 4);
    o->smem_per_cell_fp64 = camp_cell_smem_bytes(m->dm, 8);
    o->factor_updates = h.factor_updates;
    o->flops_forcing = h.flops_forcing;
    o->flops_jacobian = h.flops_jacobian;
    o->flops_factor = h.flops_factor;
    o->flops_solve = h.flops_solve;
    o->env_rh = h.rh_slot;
    o->n_electrolytes = (int32_t)h.el_phase.size();
    o->model_forcing = h.model_forcing;
    o->block_arrow = m->arrow ? 1 : 0;
    o->lanes_per_cell = m->arrow ? 0 : m->h.lanes;
    if (m->arrow) {  // the full mechanism from its one-particle template
        const camp::ArrowHost &a = m->ah;
        long long gg = 0;  // gas-gas non-zeros of the template's pattern
        for (int i = 0; i < a.n_g; i++)
            for (int q = h.rowptr[i]; q < h.rowptr[i + 1]; q++) gg += h.colidx[q] < a.n_g;
        o->n_species = m->n;
        o->n_rxn = a.Rg + a.P * a.Rp;
        o->n_env = m->n_env;
        o->n_sections = a.P;
        o->nnz_jac = (int32_t)std::min<long long>(0x7fffffff, gg + (long long)a.P * ((long long)h.colidx.size() - gg));
        const long long blk = (long long)a.n_phi * a.n_phi + 2LL * a.n_phi * a.n_c;
        o->lu_storage = (int32_t)std::min<long long>(0x7fffffff, (long long)a.P * blk + (long long)a.n_g * a.n_g);
        o->nnz_lu = o->lu_storage;
        o->rxn_map_len = 0;
        o->dense_block = a.n_g;
        o->smem_per_cell_mixed = o->smem_per_cell_fp64 = 0;
        o->factor_updates = a.flops_factor / 2;
        o->flops_forcing = a.flops_forcing;
        o->flops_jacobian = a.flops_jacobian;
        o->flops_factor = a.flops_factor;
        o->flops_solve = a.flops_solve;
        o->model_forcing = a.model_forcing;
    }
    return CAMP_OK;
}

int camp_mech_species_index(const camp_mech *m, const char *name) {
    if (!m || !name) return -1;
    if (m->arrow) {  // gas species by name; particle species as bin<p>.<name>
        const std::string s(name);
        for (int i = 0; i < m->ah.n_g; i++)
            if (m->h.species[i] == s) return i;
        const size_t dot = s.find('.');
        if (s.compare(0, 3, "bin") != 0 || dot == std::string::npos || dot == 3) return -1;
        long long p = 0;
        for (size_t k = 3; k < dot; k++) {
            if (s[k] < '0' || s[k] > '9') return -1;
            p = p * 10 + (s[k] - '0');
            if (p >= m->ah.P) return -1;
        }
        const std::string ph = "bin0" + s.substr(dot);
        for (int j = 0; j < m->ah.n_phi; j++)
            if (m->h.species[m->ah.n_g + j] == ph) return (int)(m->ah.n_g + p * m->ah.n_phi + j);
        return -1;
    }
    for (int i = 0; i < m->h.n; i++)
        if (m->h.species[i] == name) return i;
    return -1;
}

int camp_mech_structure(const camp_mech *m, int32_t *rowptr, int32_t *colidx, int32_t *rxn_map,
                        int32_t *perm, int32_t *lu_rowptr, int32_t *lu_colidx, int32_t *level_fwd,
                        int32_t *level_bwd) {
    if (!m) return fail(CAMP_E_INVAL, "NULL mechanism");
    if (m->arrow)
        return fail(CAMP_E_UNSUPPORTED, "the block-arrow form keeps one particle's structure, not a species-level one");
    const camp::HostMech &h = m->h;
    auto cp = [](int32_t *dst, const std::vector<int> &v) {
        if (dst) std::copy(v.begin(), v.end(), dst);
    };
    cp(rowptr, h.rowptr);
    cp(colidx, h.colidx);
    cp(rxn_map, h.rxn_map);
    cp(perm, h.perm);
    cp(lu_rowptr, h.lu_rowptr);
    cp(lu_colidx, h.lu_colidx);
    cp(level_fwd, h.level_fwd);
    cp(level_bwd, h.level_bwd);
    return CAMP_OK;
}

void camp_solve_opts_default(camp_solve_opts *o, int variant) {
    if (!o) return;
    o->variant = variant;
    o->persistent = -1;
    o->max_steps = 10000;
    o->cells_per_block = 0;
    o->hmin_frac = 1e-10;
    o->stats = nullptr;
    o->workspace = nullptr;
    o->step = nullptr;
}

size_t camp_workspace_bytes(void) { return 256; }

// The block-arrow form: one cell per cluster; the per-cell rows live in
// scratch allocated stream-ordered for this call (concurrent calls on other
// streams get their own).
static int arrow_solve(camp_mech *m, int64_t n_cells, double *state, const double *env, double dt, int32_t n_outer,
                       double *traj, double rtol, const double *atol, int32_t atol_len, int32_t *status,
                       const camp_solve_opts &o, cudaStream_t s) {
    const int lu = o.variant == CAMP_VARIANT_MIXED ? 4 : 8;
    const int cl = o.cells_per_block > 0 ? o.cells_per_block
                                         : (m->tuned_cpb[o.variant] > 0 ? m->tuned_cpb[o.variant] : kArrowCluster);
    int ci = -1;
    for (int k = 0; k < 5; k++)
        if (cl == (1 << k)) ci = k;
    if (ci < 0) return fail(CAMP_E_INVAL, "a block-arrow cluster holds 1, 2, 4, 8 or 16 CTAs");
    int &ncl = m->arrow_clusters[lu == 4 ? 0 : 1][ci];
    if (ncl == 0) {
        std::lock_guard<std::mutex> lk(m->mu);
        int n = 0;
        CUDA_TRY(camp_arrow_max_clusters(lu, cl, &n));
        if (n < 1) return fail(CAMP_E_UNSUPPORTED, "a block-arrow cluster does not fit on the device");
        ncl = n;
    }
    const long long clusters = std::min<long long>(ncl, n_cells);
    const size_t cell_bytes = camp_arrow_cell_bytes(m->ad, lu);
    SolveArgs a;
    a.n_cells = n_cells;
    a.state = state;
    a.env = env;
    a.dt = dt;
    a.rtol = rtol;
    a.atol = atol;
    a.atol_len = atol_len;
    a.status = status;
    a.stats = o.stats;
    a.step = o.step;
    a.max_steps = o.max_steps;
    a.hmin_frac = o.hmin_frac;
    a.cpb = 1;
    a.queue = nullptr;
    a.n_outer = n_outer;
    a.traj = traj;
    void *scratch = nullptr;
    CUDA_TRY(cudaMallocAsync(&scratch, (size_t)clusters * cell_bytes, s));
    cudaError_t e = camp_arrow_launch(m->dm, m->ad, a, lu, (char *)scratch, cell_bytes, (int)clusters, cl, s);
    cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return fail(CAMP_E_CUDA, std::string("block-arrow launch: ") + cudaGetErrorString(e));
    return CAMP_OK;
}

static int solve_impl(const camp_mech *mc, int64_t n_cells, double *state, const double *env, double dt,
                      int32_t n_outer, double *traj, double rtol, const double *atol, int32_t atol_len,
                      int32_t *status, const camp_solve_opts *opts, void *stream) {
    camp_mech *m = const_cast<camp_mech *>(mc);
    if (n_outer < 1) return fail(CAMP_E_INVAL, "n_steps must be at least 1");
    if (!m) return fail(CAMP_E_INVAL, "NULL mechanism");
    if (n_cells < 0) return fail(CAMP_E_INVAL, "n_cells < 0");
    if (n_cells == 0) return CAMP_OK;
    if (!state || !env || !atol || !status) return fail(CAMP_E_INVAL, "NULL array");
    if (!(dt > 0.0) || !(dt < 1e300)) return fail(CAMP_E_INVAL, "dt must be positive and finite");
    if (!(rtol > 0.0) || !(rtol < 1.0)) return fail(CAMP_E_INVAL, "rtol must be in (0, 1)");
    if (atol_len != 1 && atol_len != m->n) return fail(CAMP_E_INVAL, "atol_len must be 1 or n_species");
    camp_solve_opts o;
    camp_solve_opts_default(&o, opts ? opts->variant : CAMP_VARIANT_MIXED);
    if (opts) o = *opts;
    if (o.variant != CAMP_VARIANT_MIXED && o.variant != CAMP_VARIANT_FP64)
        return fail(CAMP_E_INVAL, "unknown variant");
    if (o.max_steps <= 0) o.max_steps = 10000;
    if (!(o.hmin_frac > 0.0)) o.hmin_frac = 1e-10;
    if (int rc = check_device(m)) return rc;
    if (m->arrow) return arrow_solve(m, n_cells, state, env, dt, n_outer, traj, rtol, atol, atol_len, status, o,
                                     (cudaStream_t)stream);

    const bool f32 = o.variant == CAMP_VARIANT_MIXED;
    const int smem_cell = camp_cell_smem_bytes(m->dm, f32 ? 4 : 8);
    if (o.persistent < 0)
        o.persistent = m->tuned_persistent[o.variant] >= 0 ? m->tuned_persistent[o.variant]
                                                           : (o.variant == CAMP_VARIANT_MIXED ? 1 : 0);
    auto occupancy = [&](int cpb_, int *per_sm) -> cudaError_t {
        if (m->occ[o.variant][cpb_] == 0) {
            const bool w = m->dm.n_wsec > 0;
            cudaError_t e = f32 ? (w ? camp_occupancy_f32w(m->dm, cpb_, per_sm) : camp_occupancy_f32(m->dm, cpb_, per_sm))
                                : (w ? camp_occupancy_f64w(m->dm, cpb_, per_sm) : camp_occupancy_f64(m->dm, cpb_, per_sm));
            if (e != cudaSuccess) return e;
            m->occ[o.variant][cpb_] = *per_sm > 0 ? *per_sm : -1;
        }
        *per_sm = m->occ[o.variant][cpb_] > 0 ? m->occ[o.variant][cpb_] : 0;
        return cudaSuccess;
    };
    int cpb = o.cells_per_block > 0 ? o.cells_per_block : m->tuned_cpb[o.variant];
    if (cpb <= 0) {  // most resident cells per SM, fewest cells per block on ties
        int best = 0;
        cpb = 1;
        const int max_cpb = m->h.lanes > 32 ? 1 : 4;
        for (int c2 = 1; c2 <= max_cpb; c2++) {
            if (c2 * smem_cell > kMaxSmem) break;
            int per_sm = 0;
            CUDA_TRY(occupancy(c2, &per_sm));
            if (per_sm * c2 > best) { best = per_sm * c2; cpb = c2; }
        }
    }
    cpb = std::min(cpb, 4);
    while (cpb > 1 && cpb * smem_cell > kMaxSmem) cpb--;
    if (m->h.lanes > 32) cpb = 1;  // one cell per block of threads
    if (smem_cell > kMaxSmem)
        return fail(CAMP_E_UNSUPPORTED, "one cell of this form needs more shared memory than a block may have");

    SolveArgs a;
    a.n_cells = n_cells;
    a.state = state;
    a.env = env;
    a.dt = dt;
    a.rtol = rtol;
    a.atol = atol;
    a.atol_len = atol_len;
    a.status = status;
    a.stats = o.stats;
    a.step = o.step;
    a.max_steps = o.max_steps;
    a.hmin_frac = o.hmin_frac;
    a.cpb = cpb;
    a.queue = nullptr;
    a.n_outer = n_outer;
    a.traj = traj;
    cudaStream_t s = (cudaStream_t)stream;

    long long grid;
    if (o.persistent) {
        unsigned long long *q = (unsigned long long *)o.workspace;
        if (!q) {
            std::lock_guard<std::mutex> lk(m->mu);
            if (!m->own_ws) CUDA_TRY(cudaMalloc(&m->own_ws, camp_workspace_bytes()));
            q = m->own_ws;
        }
        int per_sm = 0;
        CUDA_TRY(occupancy(cpb, &per_sm));
        if (per_sm < 1) return fail(CAMP_E_UNSUPPORTED, "kernel does not fit on an SM");
        grid = std::min<long long>((long long)per_sm * m->sm_count, (n_cells + cpb - 1) / cpb);
        CUDA_TRY(cudaMemsetAsync(q, 0, sizeof(unsigned long long), s));
        a.queue = q;
    } else {
        grid = (n_cells + cpb - 1) / cpb;
        if (grid > 0x7fffffffLL) return fail(CAMP_E_INVAL, "too many cells for one launch");
    }
    if (m->dm.n_wsec > 0)
        CUDA_TRY(f32 ? camp_launch_solve_f32w(m->dm, a, (int)grid, s) : camp_launch_solve_f64w(m->dm, a, (int)grid, s));
    else
        CUDA_TRY(f32 ? camp_launch_solve_f32(m->dm, a, (int)grid, s) : camp_launch_solve_f64(m->dm, a, (int)grid, s));
    return CAMP_OK;
}

int camp_solve(const camp_mech *m, int64_t n_cells, double *state, const double *env, double dt,
               double rtol, const double *atol, int32_t atol_len, int32_t *status,
               const camp_solve_opts *opts, void *stream) {
    CampRange range_("camp_solve");
    return solve_impl(m, n_cells, state, env, dt, 1, nullptr, rtol, atol, atol_len, status, opts, stream);
}

int camp_solve_sequence(const camp_mech *m, int64_t n_cells, double *state, const double *env, double dt,
                        int32_t n_steps, double *trajectory, double rtol, const double *atol,
                        int32_t atol_len, int32_t *status, const camp_solve_opts *opts, void *stream) {
    CampRange range_("camp_solve_sequence");
    return solve_impl(m, n_cells, state, env, dt, n_steps, trajectory, rtol, atol, atol_len, status, opts,
                      stream);
}

int camp_solve_host(const camp_mech *mc, int64_t n_cells, double *state, const double *env,
                    double dt, double rtol, const double *atol, int32_t atol_len, int32_t *status,
                    const camp_solve_opts *opts, void *stream) {
    CampRange range_("camp_solve_host");
    camp_mech *m = const_cast<camp_mech *>(mc);
    if (!m) return fail(CAMP_E_INVAL, "NULL mechanism");
    if (n_cells <= 0) return n_cells == 0 ? CAMP_OK : fail(CAMP_E_INVAL, "n_cells < 0");
    if (!state || !env || !atol || !status) return fail(CAMP_E_INVAL, "NULL array");
    if (atol_len != 1 && atol_len != m->n) return fail(CAMP_E_INVAL, "atol_len must be 1 or n_species");
    if (int rc = check_device(m)) return rc;
    const size_t n = m->n, ne = m->n_env;
    const size_t b_state = (size_t)n_cells * n * 8, b_env = (size_t)n_cells * ne * 8;
    const size_t b_stat = ((size_t)n_cells * 4 + 15) & ~(size_t)15, b_atol = (n * 8 + 15) & ~(size_t)15;
    const size_t b_stats = (size_t)n_cells * 4 * CAMP_NSTATS;
    int32_t *host_stats = opts ? opts->stats : nullptr;
    double *host_step = opts ? opts->step : nullptr;
    const size_t b_step = host_step ? (((size_t)n_cells * 8 + 15) & ~(size_t)15) : 0;
    const size_t need = b_state + b_env + b_stat + b_atol + b_step + (host_stats ? b_stats : 0);
    std::lock_guard<std::mutex> lk(m->stage_mu);
    if (m->stage_bytes < need) {
        if (m->stage) cudaFree(m->stage);
        m->stage = nullptr;
        m->stage_bytes = 0;
        CUDA_TRY(cudaMalloc(&m->stage, need));
        m->stage_bytes = need;
    }
    char *base = (char *)m->stage;
    double *d_state = (double *)base;
    double *d_env = (double *)(base + b_state);
    int32_t *d_status = (int32_t *)(base + b_state + b_env);
    double *d_atol = (double *)(base + b_state + b_env + b_stat);
    double *d_step = host_step ? (double *)(base + b_state + b_env + b_stat + b_atol) : nullptr;
    int32_t *d_stats = host_stats ? (int32_t *)(base + b_state + b_env + b_stat + b_atol + b_step) : nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    CUDA_TRY(cudaMemcpyAsync(d_state, state, b_state, cudaMemcpyHostToDevice, s));
    if (host_step) CUDA_TRY(cudaMemcpyAsync(d_step, host_step, (size_t)n_cells * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_env, env, b_env, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_atol, atol, (size_t)atol_len * 8, cudaMemcpyHostToDevice, s));
    camp_solve_opts o;
    camp_solve_opts_default(&o, opts ? opts->variant : CAMP_VARIANT_MIXED);
    if (opts) o = *opts;
    o.stats = d_stats;
    o.step = d_step;
    o.workspace = nullptr;
    int rc = camp_solve(m, n_cells, d_state, d_env, dt, rtol, d_atol, atol_len, d_status, &o, stream);
    if (rc != CAMP_OK) return rc;
    CUDA_TRY(cudaMemcpyAsync(state, d_state, b_state, cudaMemcpyDeviceToHost, s));
    if (host_step) CUDA_TRY(cudaMemcpyAsync(host_step, d_step, (size_t)n_cells * 8, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaMemcpyAsync(status, d_status, (size_t)n_cells * 4, cudaMemcpyDeviceToHost, s));
    if (host_stats)
        CUDA_TRY(cudaMemcpyAsync(host_stats, d_stats, b_stats, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return CAMP_OK;
}

int camp_solve_batch(const camp_group *groups, int32_t n_groups, double dt, double rtol,
                     const camp_solve_opts *opts, void *stream) {
    CampRange range_("camp_solve_batch");
    if (!groups || n_groups < 0 || n_groups > CAMP_MAX_GROUPS) return fail(CAMP_E_INVAL, "bad group count");
    if (n_groups == 0) return CAMP_OK;
    // estimated work of one cell (f flops + LU solve flops + vector work),
    // costliest cells first: each group's persistent grid holds the SMs
    // until its counter runs dry, so the groups run one after the other and
    // the last group's cells make the batch's tail -- best the shortest ones
    int order[CAMP_MAX_GROUPS];
    double work[CAMP_MAX_GROUPS];
    for (int g = 0; g < n_groups; g++) {
        if (!groups[g].mech) return fail(CAMP_E_INVAL, "NULL mechanism in group");
        const camp::HostMech &h = groups[g].mech->h;
        work[g] = groups[g].mech->arrow
                      ? (double)(groups[g].mech->ah.flops_forcing + groups[g].mech->ah.flops_solve +
                                 20LL * groups[g].mech->n)
                      : (double)(h.flops_forcing + h.flops_solve + 20 * h.n);
        order[g] = g;
    }
    std::sort(order, order + n_groups, [&](int a, int b) { return work[a] > work[b]; });
    cudaStream_t parent = (cudaStream_t)stream;
    thread_local cudaStream_t forks[CAMP_MAX_GROUPS] = {};
    thread_local cudaEvent_t ev_fork = nullptr, ev_join[CAMP_MAX_GROUPS] = {};
    thread_local int fork_dev = -1;
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (fork_dev != dev) {
        for (int g = 0; g < CAMP_MAX_GROUPS; g++) {
            CUDA_TRY(cudaStreamCreateWithFlags(&forks[g], cudaStreamNonBlocking));
            CUDA_TRY(cudaEventCreateWithFlags(&ev_join[g], cudaEventDisableTiming));
        }
        CUDA_TRY(cudaEventCreateWithFlags(&ev_fork, cudaEventDisableTiming));
        fork_dev = dev;
    }
    CUDA_TRY(cudaEventRecord(ev_fork, parent));
    int rc = CAMP_OK;
    for (int i = 0; i < n_groups; i++) {
        const camp_group &gr = groups[order[i]];
        CUDA_TRY(cudaStreamWaitEvent(forks[i], ev_fork, 0));
        camp_solve_opts o;
        camp_solve_opts_default(&o, opts ? opts->variant : CAMP_VARIANT_MIXED);
        if (opts) o = *opts;
        o.stats = gr.stats;
        o.workspace = gr.workspace;
        o.step = gr.step;
        if (o.persistent < 0) o.persistent = 1;
        if (!o.workspace && n_groups > 1 && o.persistent)
            return fail(CAMP_E_INVAL, "each group of a multi-group persistent solve needs its own workspace");
        rc = camp_solve(gr.mech, gr.n_cells, gr.state, gr.env, dt, rtol, gr.atol, gr.atol_len, gr.status,
                        &o, forks[i]);
        CUDA_TRY(cudaEventRecord(ev_join[i], forks[i]));
        CUDA_TRY(cudaStreamWaitEvent(parent, ev_join[i], 0));
        if (rc != CAMP_OK) return rc;
    }
    return CAMP_OK;
}

int camp_solve_batch_host(const camp_group *groups, int32_t n_groups, double dt, double rtol,
                          const camp_solve_opts *opts, void *stream) {
    CampRange range_("camp_solve_batch_host");
    if (!groups || n_groups < 0 || n_groups > CAMP_MAX_GROUPS) return fail(CAMP_E_INVAL, "bad group count");
    if (n_groups == 0) return CAMP_OK;
    static std::mutex mu;
    static void *stage[64] = {};
    static size_t stage_bytes[64] = {};
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(CAMP_E_INVAL, "device ordinal out of range");
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    struct Part { size_t state, env, atol, status, stats, step, ws; };
    Part part[CAMP_MAX_GROUPS];
    size_t need = 0;
    for (int g = 0; g < n_groups; g++) {
        const camp_group &gr = groups[g];
        if (!gr.mech) return fail(CAMP_E_INVAL, "NULL mechanism in group");
        if (gr.n_cells < 0) return fail(CAMP_E_INVAL, "n_cells < 0");
        if (gr.n_cells > 0 && (!gr.state || !gr.env || !gr.atol || !gr.status))
            return fail(CAMP_E_INVAL, "NULL array in group");
        if (gr.atol_len != 1 && gr.atol_len != gr.mech->n) return fail(CAMP_E_INVAL, "atol_len must be 1 or n_species");
        if (int rc = check_device(gr.mech)) return rc;
        const size_t C = (size_t)gr.n_cells;
        Part &p = part[g];
        p.state = need; need += al(C * gr.mech->n * 8);
        p.env = need; need += al(C * gr.mech->n_env * 8);
        p.atol = need; need += al((size_t)gr.atol_len * 8);
        p.status = need; need += al(C * 4);
        p.stats = need; need += gr.stats ? al(C * 4 * CAMP_NSTATS) : 0;
        p.step = need; need += gr.step ? al(C * 8) : 0;
        p.ws = need; need += al(camp_workspace_bytes());
    }
    std::lock_guard<std::mutex> lk(mu);
    if (stage_bytes[dev] < need) {
        if (stage[dev]) cudaFree(stage[dev]);
        stage[dev] = nullptr;
        stage_bytes[dev] = 0;
        CUDA_TRY(cudaMalloc(&stage[dev], need));
        stage_bytes[dev] = need;
    }
    char *base = (char *)stage[dev];
    cudaStream_t s = (cudaStream_t)stream;
    camp_group dg[CAMP_MAX_GROUPS];
    // once a copy is enqueued, every return waits for the stream: the next
    // call may reuse the buffer as soon as the lock is released
    auto drain = [&](int rc) {
        cudaStreamSynchronize(s);
        return rc;
    };
    for (int g = 0; g < n_groups; g++) {
        const camp_group &gr = groups[g];
        const Part &p = part[g];
        const size_t C = (size_t)gr.n_cells;
        dg[g] = gr;
        dg[g].state = (double *)(base + p.state);
        dg[g].env = (const double *)(base + p.env);
        dg[g].atol = (const double *)(base + p.atol);
        dg[g].status = (int32_t *)(base + p.status);
        dg[g].stats = gr.stats ? (int32_t *)(base + p.stats) : nullptr;
        dg[g].step = gr.step ? (double *)(base + p.step) : nullptr;
        dg[g].workspace = base + p.ws;
        if (C == 0) continue;
        cudaError_t e = cudaMemcpyAsync(dg[g].state, gr.state, C * gr.mech->n * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((void *)dg[g].env, gr.env, C * gr.mech->n_env * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((void *)dg[g].atol, gr.atol, (size_t)gr.atol_len * 8, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && gr.step) e = cudaMemcpyAsync(dg[g].step, gr.step, C * 8, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess)
            return drain(fail(CAMP_E_CUDA, std::string("staging copy: ") + cudaGetErrorString(e)));
    }
    int rc = camp_solve_batch(dg, n_groups, dt, rtol, opts, stream);
    if (rc != CAMP_OK) return drain(rc);
    for (int g = 0; g < n_groups; g++) {
        const camp_group &gr = groups[g];
        const size_t C = (size_t)gr.n_cells;
        if (C == 0) continue;
        cudaError_t e = cudaMemcpyAsync(gr.state, dg[g].state, C * gr.mech->n * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(gr.status, dg[g].status, C * 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && gr.stats)
            e = cudaMemcpyAsync(gr.stats, dg[g].stats, C * 4 * CAMP_NSTATS, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && gr.step) e = cudaMemcpyAsync(gr.step, dg[g].step, C * 8, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return drain(fail(CAMP_E_CUDA, std::string("result copy: ") + cudaGetErrorString(e)));
    }
    CUDA_TRY(cudaStreamSynchronize(s));
    return CAMP_OK;
}

int camp_autotune(camp_mech *m, int64_t n_cells, const double *state, const double *env, double dt,
                  double rtol, const double *atol, int32_t atol_len, int32_t variant, int32_t *best_cpb,
                  int32_t *best_persistent, double *ms_best, void *stream) {
    CampRange range_("camp_autotune");
    if (!m || n_cells <= 0 || !state || !env || !atol) return fail(CAMP_E_INVAL, "bad argument");
    if (variant != CAMP_VARIANT_MIXED && variant != CAMP_VARIANT_FP64) return fail(CAMP_E_INVAL, "unknown variant");
    if (int rc = check_device(m)) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t bytes = (size_t)n_cells * m->n * 8;
    double *work = nullptr;
    int32_t *status = nullptr;
    CUDA_TRY(cudaMallocAsync((void **)&work, bytes, s));
    CUDA_TRY(cudaMallocAsync((void **)&status, (size_t)n_cells * 4, s));
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    // the block-arrow form: CTAs per cluster 2, 4, 8, 16 (one launch shape
    // otherwise); the others: cells per block 1-4 x static / persistent grid,
    // on each cell shape the mechanism can take (129-256 species: one warp
    // or 64 threads a cell, camp_alt_lanes), the tables rebuilt for each
    const int cpbs[4] = {1, 2, 3, 4}, clusters[4] = {2, 4, 8, 16};
    const int def_lanes = camp_cell_lanes(m->h.n), alt = m->arrow ? 0 : camp_alt_lanes(m->h.n);
    const int lane_opts[2] = {m->h.lanes, m->h.lanes == def_lanes ? alt : def_lanes};
    float best = 1e30f;
    int bc = 1, bp = 1, bl = m->h.lanes, rc = CAMP_OK;
    for (int li = 0; li < (alt ? 2 : 1) && rc == CAMP_OK; li++) {
        if (li > 0) rc = mech_relane(m, lane_opts[li]);
        if (rc != CAMP_OK) break;
        int cand_choice[8], cand_pers[8], nc = 0;
        for (int pers = m->arrow ? 1 : 0; pers <= 1; pers++)
            for (int ci = 0; ci < 4; ci++) {
                const int smem_cell = camp_cell_smem_bytes(m->dm, variant == CAMP_VARIANT_MIXED ? 4 : 8);
                if (!m->arrow && cpbs[ci] * smem_cell > kMaxSmem) continue;
                if (!m->arrow && cpbs[ci] > 1 && m->h.lanes > 32) continue;  // a block is one cell
                cand_choice[nc] = m->arrow ? clusters[ci] : cpbs[ci];
                cand_pers[nc++] = pers;
            }
        // one untimed solve first (clocks ramp up and tables reach the
        // caches), then two sweeps over the candidates, each keeping its
        // faster time, so that a slow stretch of the GPU does not decide
        float t[8];
        for (int i = 0; i < nc; i++) t[i] = 1e30f;
        for (int sweep = -1; sweep < 2 && rc == CAMP_OK; sweep++)
            for (int i = 0; i < (sweep < 0 ? 1 : nc) && rc == CAMP_OK; i++) {
                camp_solve_opts o;
                camp_solve_opts_default(&o, variant);
                o.persistent = cand_pers[i];
                o.cells_per_block = cand_choice[i];
                if (cudaMemcpyAsync(work, state, bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess) rc = CAMP_E_CUDA;
                cudaEventRecord(e0, s);
                if (rc == CAMP_OK) rc = camp_solve(m, n_cells, work, env, dt, rtol, atol, atol_len, status, &o, s);
                cudaEventRecord(e1, s);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = CAMP_E_CUDA;
                float ms = 0.f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (sweep >= 0 && ms < t[i]) t[i] = ms;
            }
        for (int i = 0; i < nc && rc == CAMP_OK; i++)
            if (t[i] < best) { best = t[i]; bc = cand_choice[i]; bp = cand_pers[i]; bl = m->h.lanes; }
    }
    if (rc == CAMP_OK && bl != m->h.lanes) rc = mech_relane(m, bl);
    cudaFreeAsync(work, s);
    cudaFreeAsync(status, s);
    cudaStreamSynchronize(s);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != CAMP_OK) return rc;
    m->tuned_cpb[variant] = bc;
    m->tuned_persistent[variant] = bp;
    if (best_cpb) *best_cpb = bc;
    if (best_persistent) *best_persistent = bp;
    if (ms_best) *ms_best = best;
    return CAMP_OK;
}

int camp_rate_constants(const camp_mech *m, int64_t n_cells, const double *env, double *kf,
                        double *kr, void *stream) {
    if (!m || n_cells < 0 || (n_cells && (!env || !kf || !kr))) return fail(CAMP_E_INVAL, "bad argument");
    if (!n_cells) return CAMP_OK;
    if (int rc = check_device(m)) return rc;
    if (m->arrow) return fail(CAMP_E_UNSUPPORTED, "the block-arrow form keeps rate constants per particle inside the solve");
    CUDA_TRY(camp_launch_rates(m->dm, n_cells, env, kf, kr, (cudaStream_t)stream));
    return CAMP_OK;
}

int camp_forcing(const camp_mech *m, int64_t n_cells, const double *state, const double *env,
                 double *f, void *stream) {
    if (!m || n_cells < 0 || (n_cells && (!state || !env || !f))) return fail(CAMP_E_INVAL, "bad argument");
    if (!n_cells) return CAMP_OK;
    if (n_cells > 0x7fffffffLL) return fail(CAMP_E_INVAL, "too many cells");
    if (int rc = check_device(m)) return rc;
    if (m->arrow) {
        CUDA_TRY(camp_arrow_forcing(m->dm, m->ad, n_cells, state, env, f, (cudaStream_t)stream));
        return CAMP_OK;
    }
    CUDA_TRY(camp_launch_forcing(m->dm, n_cells, state, env, f, (cudaStream_t)stream));
    return CAMP_OK;
}

int camp_jacobian(const camp_mech *m, int64_t n_cells, const double *state, const double *env,
                  double *jac, int32_t variant, void *stream) {
    if (!m || n_cells < 0 || (n_cells && (!state || !env || !jac))) return fail(CAMP_E_INVAL, "bad argument");
    if (variant != CAMP_VARIANT_MIXED && variant != CAMP_VARIANT_FP64) return fail(CAMP_E_INVAL, "unknown variant");
    if (!n_cells) return CAMP_OK;
    if (n_cells > 0x7fffffffLL) return fail(CAMP_E_INVAL, "too many cells");
    if (int rc = check_device(m)) return rc;
    if (m->arrow) return fail(CAMP_E_UNSUPPORTED, "the block-arrow form assembles and factors inside the solve");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->dm.n_wsec > 0)
        CUDA_TRY(variant == CAMP_VARIANT_MIXED ? camp_launch_jacobian_f32w(m->dm, n_cells, state, env, jac, s)
                                               : camp_launch_jacobian_f64w(m->dm, n_cells, state, env, jac, s));
    else
        CUDA_TRY(variant == CAMP_VARIANT_MIXED ? camp_launch_jacobian_f32(m->dm, n_cells, state, env, jac, s)
                                               : camp_launch_jacobian_f64(m->dm, n_cells, state, env, jac, s));
    return CAMP_OK;
}

int camp_lu_solve(const camp_mech *m, int64_t n_cells, const double *state, const double *env,
                  double gamma, const double *b, double *x, int32_t *status, int32_t variant,
                  void *stream) {
    if (!m || n_cells < 0 || (n_cells && (!state || !env || !b || !x || !status)))
        return fail(CAMP_E_INVAL, "bad argument");
    if (variant != CAMP_VARIANT_MIXED && variant != CAMP_VARIANT_FP64) return fail(CAMP_E_INVAL, "unknown variant");
    if (!n_cells) return CAMP_OK;
    if (n_cells > 0x7fffffffLL) return fail(CAMP_E_INVAL, "too many cells");
    if (int rc = check_device(m)) return rc;
    if (m->arrow) return fail(CAMP_E_UNSUPPORTED, "the block-arrow form assembles and factors inside the solve");
    cudaStream_t s = (cudaStream_t)stream;
    if (m->dm.n_wsec > 0)
        CUDA_TRY(variant == CAMP_VARIANT_MIXED
                     ? camp_launch_lu_solve_f32w(m->dm, n_cells, state, env, gamma, b, x, status, s)
                     : camp_launch_lu_solve_f64w(m->dm, n_cells, state, env, gamma, b, x, status, s));
    else
        CUDA_TRY(variant == CAMP_VARIANT_MIXED
                     ? camp_launch_lu_solve_f32(m->dm, n_cells, state, env, gamma, b, x, status, s)
                     : camp_launch_lu_solve_f64(m->dm, n_cells, state, env, gamma, b, x, status, s));
    return CAMP_OK;
}

}  // extern "C"
