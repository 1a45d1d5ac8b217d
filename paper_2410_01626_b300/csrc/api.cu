// C ABI of the fmmcph library: handle lifecycle, argument validation, buffers.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>
#include <algorithm>
#include <map>
#include <memory>
#include <mutex>
#include <atomic>

#include "fmm_internal.h"
#include "operators.h"

using namespace fmmcph;

struct fmm_handle {
    Handle h;
};

// Allocation-failure injection: > 0 counts down the library's device allocations; the one that
// brings it to zero fails as if the device were out of memory (no cudaMalloc is attempted).
static std::atomic<int> g_fail_alloc_in{0};

cudaError_t fmmcph::device_alloc(void** p, size_t bytes) {
    int k = g_fail_alloc_in.load();
    while (k > 0 && !g_fail_alloc_in.compare_exchange_weak(k, k - 1)) {
    }
    if (k == 1) {
        *p = nullptr;
        return cudaErrorMemoryAllocation;
    }
    return cudaMalloc(p, bytes);
}

namespace {

thread_local char g_last_error[256] = "";

// Records the failing call and CUDA's message for fmm_last_error(); returns FMM_ERR_CUDA.
fmm_status cuda_fail(const char* what, cudaError_t e) {
    snprintf(g_last_error, sizeof(g_last_error), "%s: %s", what, cudaGetErrorString(e));
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
}

template <class T>
fmm_status dalloc(T** p, size_t count) {
    *p = nullptr;
    if (count == 0) count = 1;
    if (device_alloc((void**)p, sizeof(T) * count) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return FMM_ERR_OOM;
    }
    return FMM_OK;
}

template <class T>
void dfree(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

void free_atoms(Handle& h) {
    dfree(h.qA);
    dfree(h.qB);
    dfree(h.site);
    dfree(h.key);
    dfree(h.kA);
    dfree(h.kB);
    dfree(h.vA);
    dfree(h.vB);
    dfree(h.inv);
    dfree(h.pos);
    dfree(h.dq);
    dfree(h.phis);
    dfree(h.near);
    dfree(h.near_items);
    h.near_items_cap = 0;
    dfree(h.qC);
    dfree(h.qD);
    dfree(h.dqt);
    h.perm = nullptr;
    h.sorted_key = nullptr;
    h.cap = 0;
}

void free_all(Handle& h) {
    m2l_tc_free(&h);  // every error path of fmm_create after m2l_tc_setup releases its state too
    free_atoms(h);
    dfree(h.T);
    dfree(h.A);
    dfree(h.B);
    dfree(h.B2);
    dfree(h.Ad);
    dfree(h.Lam);
    translate_free(h.m2m_tc);
    translate_free(h.l2l_tc);
    dfree(h.tiles);
    dfree(h.bricks);
    dfree(h.m2l_part);
    dfree(h.M);
    dfree(h.L);
    dfree(h.lam);
    dfree(h.site_ptr);
    dfree(h.site_atoms);
    dfree(h.start);
    dfree(h.count);
    dfree(h.leafcnt);
    dfree(h.epart);
    dfree(h.leafmom);
    dfree(h.hi_coef);
    dfree(h.hi_site);
    dfree(h.hi_g);
    dfree(h.root);
    dfree(h.status);
    dfree(h.work);
    for (int i = 0; i < 2; ++i) {
        dfree(h.hx_dev[i]);
        dfree(h.hF_dev[i]);
        dfree(h.hdV_dev[i]);
        dfree(h.hE_dev[i]);
    }
    if (h.ev_valid) {
        for (auto& e : h.ev) cudaEventDestroy(e);
    }
    h.ev_valid = false;
    if (h.fork_ev) cudaEventDestroy(h.fork_ev);
    if (h.join_ev) cudaEventDestroy(h.join_ev);
    if (h.eval_ev) cudaEventDestroy(h.eval_ev);
    h.eval_ev = nullptr;
    h.eval_ev_valid = false;
    for (cudaEvent_t* e : {&h.m2m_ev, &h.side_ev}) {
        if (*e) cudaEventDestroy(*e);
        *e = nullptr;
    }
    if (h.chain) cudaStreamDestroy(h.chain);
    if (h.side) cudaStreamDestroy(h.side);
    h.fork_ev = h.join_ev = nullptr;
    h.chain = h.side = nullptr;
    for (auto& g : h.g_slot) {
        if (g.exec) cudaGraphExecDestroy(g.exec);
        g.exec = nullptr;
    }
    if (h.gcap) cudaStreamDestroy(h.gcap);
    h.gcap = nullptr;
    for (int i = 0; i < 2; ++i) {
        if (h.hx_ev[i]) cudaEventDestroy(h.hx_ev[i]);
        if (h.hfree_ev[i]) cudaEventDestroy(h.hfree_ev[i]);
        h.hx_ev[i] = h.hfree_ev[i] = nullptr;
    }
    if (h.h2d) cudaStreamDestroy(h.h2d);
    h.h2d = nullptr;
}

inline cudaStream_t S(void* s) { return (cudaStream_t)s; }

fmm_status cuda_ok(cudaError_t e) {
    if (e == cudaSuccess) return FMM_OK;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? FMM_ERR_OOM : FMM_ERR_CUDA;
}

}  // namespace

// Host-built operator banks depend only on (p, periodic); handles in one process share them.
struct HostOps {
    std::vector<float> T, Trm, A, B, B2;
    std::vector<double> Ad, Lam;
};

static std::shared_ptr<const HostOps> host_ops(int p, int periodic, bool want_rowmajor) {
    static std::mutex mu;
    static std::map<std::pair<int, int>, std::shared_ptr<HostOps>> cache;
    const int nc = ncoef(p), ncp = ncoef_padded(p);
    std::lock_guard<std::mutex> lock(mu);
    auto& slot = cache[{p, periodic}];
    if (slot && (!want_rowmajor || !slot->Trm.empty())) return slot;
    auto o = std::make_shared<HostOps>();
    std::vector<double> op((size_t)nc * nc);
    o->T.assign((size_t)kNumOps * ncp * ncp, 0.f);
    o->Trm.assign((size_t)kNumOps * nc * nc, 0.f);
    for (int ox = -3; ox <= 3; ++ox)
        for (int oy = -3; oy <= 3; ++oy)
            for (int oz = -3; oz <= 3; ++oz) {
                if (std::max(std::abs(ox), std::max(std::abs(oy), std::abs(oz))) < 2) continue;
                const int oo[3] = {ox, oy, oz};
                op_m2l(p, oo, op.data());
                float* dst = o->T.data() + (size_t)op_index(ox, oy, oz) * ncp * ncp;
                for (int j = 0; j < nc; ++j)
                    for (int k = 0; k < nc; ++k) dst[(size_t)k * ncp + j] = (float)op[(size_t)j * nc + k];
                for (size_t e = 0; e < (size_t)nc * nc; ++e)
                    o->Trm[(size_t)op_index(ox, oy, oz) * nc * nc + e] = (float)op[e];
            }
    o->A.assign((size_t)8 * ncp * ncp, 0.f);
    o->B.assign((size_t)8 * ncp * ncp, 0.f);
    o->B2.assign((size_t)8 * ncp * ncp, 0.f);
    o->Ad.resize((size_t)8 * nc * nc);
    for (int c = 0; c < 8; ++c) {
        op_m2m(p, c, op.data());
        std::memcpy(o->Ad.data() + (size_t)c * nc * nc, op.data(), sizeof(double) * nc * nc);
        for (int j = 0; j < nc; ++j)
            for (int k = 0; k < nc; ++k) o->A[((size_t)c * ncp + k) * ncp + j] = (float)op[(size_t)j * nc + k];
        op_l2l(p, c, op.data());
        for (int j = 0; j < nc; ++j)
            for (int k = 0; k < nc; ++k) {
                o->B[((size_t)c * ncp + k) * ncp + j] = (float)op[(size_t)j * nc + k];
                o->B2[(size_t)k * 8 * ncp + c * ncp + j] = (float)op[(size_t)j * nc + k];
            }
    }
    if (periodic) {
        o->Lam.resize((size_t)nc * nc);
        op_lattice(p, o->Lam.data());
    }
    slot = o;
    return slot;
}

extern "C" {

const char* fmm_last_error(void) { return g_last_error; }

const char* fmm_error_string(fmm_status s) {
    switch (s) {
        case FMM_OK: return "ok";
        case FMM_ERR_ARG: return "invalid argument";
        case FMM_ERR_DOMAIN: return "atom outside the open box";
        case FMM_ERR_CUDA: return "CUDA runtime error";
        case FMM_ERR_OOM: return "device allocation failed";
        case FMM_ERR_TIMEOUT: return "bounded device wait expired";
        case FMM_ERR_STATE: return "call order violated";
    }
    return "unknown status";
}

fmm_status fmm_host_operator(int kind, int p, const int* o, double* out) {
    if (p < 1 || p > FMM_MAX_P || !out) return FMM_ERR_ARG;
    switch (kind) {
        case 0: {
            if (!o) return FMM_ERR_ARG;
            int mx = std::max(std::abs(o[0]), std::max(std::abs(o[1]), std::abs(o[2])));
            if (mx < 2 || mx > 3) return FMM_ERR_ARG;
            op_m2l(p, o, out);
            return FMM_OK;
        }
        case 1:
        case 2:
            if (!o || o[0] < 0 || o[0] > 7) return FMM_ERR_ARG;
            if (kind == 1) op_m2m(p, o[0], out);
            else op_l2l(p, o[0], out);
            return FMM_OK;
        case 3:
            op_lattice(p, out);
            return FMM_OK;
    }
    return FMM_ERR_ARG;
}

fmm_status fmm_host_regular(int p, const double* u, double* out) {
    if (p < 0 || p > 2 * FMM_MAX_P || !u || !out) return FMM_ERR_ARG;
    regular_real_hat(p, u, out);
    return FMM_OK;
}

fmm_status fmm_create(const fmm_box* box, int periodic, int p, int depth, const fmm_options* opt,
                      fmm_handle** out) {
    if (!out) return FMM_ERR_ARG;
    *out = nullptr;
    if (!box || !(box->edge > 0.0) || !std::isfinite(box->edge)) return FMM_ERR_ARG;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(box->origin[a])) return FMM_ERR_ARG;
    if (periodic != 0 && periodic != 1) return FMM_ERR_ARG;
    if (p < 1 || p > FMM_MAX_P || depth < 0 || depth > kMaxDepth) return FMM_ERR_ARG;
    int precision = FMM_FP32, interpolation = FMM_INTERP_CHARGE;
    int m2l_rows = 0, p2p_warps = 0;
    double ke = 138.935458;
    if (opt) {
        for (int r : opt->reserved)
            if (r != 0) return FMM_ERR_ARG;
        if (opt->precision < FMM_FP32 || opt->precision > FMM_MIXED_FP16) return FMM_ERR_ARG;
        if (opt->interpolation != FMM_INTERP_CHARGE && opt->interpolation != FMM_INTERP_HAMILTONIAN)
            return FMM_ERR_ARG;
        if (!m2l_tile_rows_ok(opt->m2l_tile_rows)) return FMM_ERR_ARG;
        if (opt->p2p_leaves_per_block != 0 && opt->p2p_leaves_per_block != 1 && opt->p2p_leaves_per_block != 2 &&
            opt->p2p_leaves_per_block != 4)
            return FMM_ERR_ARG;
        precision = opt->precision;
        interpolation = opt->interpolation;
        m2l_rows = opt->m2l_tile_rows;
        p2p_warps = opt->p2p_leaves_per_block;
        if (opt->coulomb_k > 0.0) ke = opt->coulomb_k;
    }
    fmm_handle* H = new (std::nothrow) fmm_handle();
    if (!H) return FMM_ERR_OOM;
    Handle& h = H->h;
    cudaGetDevice(&h.device);
    h.box = *box;
    h.periodic = periodic;
    h.p = p;
    h.depth = depth;
    h.nc = ncoef(p);
    h.ncp = ncoef_padded(p);
    h.precision = precision;
    h.m2l_rows = m2l_rows;
    h.p2p_warps = p2p_warps > 0 ? p2p_warps : 1;
    h.hamiltonian = interpolation == FMM_INTERP_HAMILTONIAN;
    h.ke = ke;
    h.s_bin = std::ldexp(1.0, depth) / box->edge;
    h.lmin = periodic ? 1 : 2;
    if (precision != FMM_FP32 && !m2l_tc_supported(&h)) {  // no silent fallback to another precision
        delete H;
        return FMM_ERR_ARG;
    }
    upload_constants(p);
    near_configure(&h);

    const int nc = h.nc, ncp = h.ncp;
    fmm_status st = FMM_OK;
    // ---- operators (host banks cached per (p, periodic)) ----
    {
        const std::shared_ptr<const HostOps> ops = host_ops(p, periodic, precision != FMM_FP32);
        if ((st = dalloc(&h.T, ops->T.size())) || (st = dalloc(&h.A, ops->A.size())) ||
            (st = dalloc(&h.B, ops->B.size())) || (st = dalloc(&h.B2, ops->B2.size())) ||
            (st = dalloc(&h.Ad, ops->Ad.size())) || (periodic && (st = dalloc(&h.Lam, ops->Lam.size())))) {
            free_all(h);
            delete H;
            return st;
        }
        cudaMemcpy(h.T, ops->T.data(), sizeof(float) * ops->T.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(h.A, ops->A.data(), sizeof(float) * ops->A.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(h.B, ops->B.data(), sizeof(float) * ops->B.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(h.B2, ops->B2.data(), sizeof(float) * ops->B2.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(h.Ad, ops->Ad.data(), sizeof(double) * ops->Ad.size(), cudaMemcpyHostToDevice);
        if (periodic) cudaMemcpy(h.Lam, ops->Lam.data(), sizeof(double) * ops->Lam.size(), cudaMemcpyHostToDevice);
        if (h.hamiltonian && periodic) {
            // the harmonic remainder h of the periodic pair potential: the lattice operator's
            // response to a unit charge at the root centre, i.e. its first column
            std::vector<float> hc(ncp, 0.f);
            for (int j = 0; j < nc; ++j) hc[j] = (float)ops->Lam[(size_t)j * nc];
            if ((st = dalloc(&h.hi_coef, ncp))) {
                free_all(h);
                delete H;
                return st;
            }
            cudaMemcpy(h.hi_coef, hc.data(), sizeof(float) * ncp, cudaMemcpyHostToDevice);
        }
        if (precision != FMM_FP32) {
            h.lvl_off.assign(depth + 2, 0);
            long a2 = 0;
            for (int l = 0; l <= depth; ++l) {
                h.lvl_off[l] = a2;
                a2 += 1L << (3 * l);
            }
            int e = m2l_tc_setup(&h, ops->Trm);
            if (e == FMM_OK) {  // M2M [ncp][8 ncp] and L2L [8 ncp][ncp] as row-major W[m][k]
                std::vector<float> W((size_t)8 * ncp * ncp);
                for (int c = 0; c < 8; ++c)
                    for (int k = 0; k < ncp; ++k)
                        for (int j = 0; j < ncp; ++j)
                            W[(size_t)j * 8 * ncp + c * ncp + k] = ops->A[((size_t)c * ncp + k) * ncp + j];
                h.m2m_tc = translate_pack(W, ncp, 8 * ncp);
                for (int k = 0; k < ncp; ++k)
                    for (int cj = 0; cj < 8 * ncp; ++cj) W[(size_t)cj * ncp + k] = ops->B2[(size_t)k * 8 * ncp + cj];
                h.l2l_tc = translate_pack(W, 8 * ncp, ncp);
                if (!h.m2m_tc.dev || !h.l2l_tc.dev) e = FMM_ERR_OOM;
                translate_configure();
            }
            if (e != FMM_OK) {
                m2l_tc_free(&h);
                free_all(h);
                delete H;
                return (fmm_status)e;
            }
        }
    }
    // ---- tree storage and work lists ----
    h.lvl_off.assign(depth + 2, 0);
    long acc = 0;
    for (int l = 0; l <= depth; ++l) {
        h.lvl_off[l] = acc;
        acc += 1L << (3 * l);
    }
    h.lvl_off[depth + 1] = acc;
    h.nbox_total = acc;
    std::vector<M2LTile> tiles;
    for (int l = h.lmin; l <= depth; ++l) {
        const int np = 1 << (3 * (l - 1));
        for (int c = 0; c < 8; ++c)
            for (int p0 = 0; p0 < np; p0 += 16) tiles.push_back({l, c, p0, std::min(16, np - p0)});
    }
    h.ntiles = (int)tiles.size();
    std::vector<F32Brick> bricks;
    if (precision == FMM_FP32 && ncp <= 128) f32_bricks(h.lmin, depth, bricks);
    h.nbricks = (int)bricks.size();
    const long nleaf = 1L << (3 * depth);
    if ((st = dalloc(&h.M, (size_t)acc * ncp)) || (st = dalloc(&h.L, (size_t)acc * ncp)) ||
        (st = dalloc(&h.tiles, tiles.size())) || (st = dalloc(&h.bricks, bricks.size())) ||
        (!bricks.empty() && (st = dalloc(&h.m2l_part, 8L * acc * ncp))) || (st = dalloc(&h.start, nleaf)) ||
        (st = dalloc(&h.count, nleaf)) || (st = dalloc(&h.leafcnt, leafcnt_words(nleaf))) || (st = dalloc(&h.epart, nleaf)) ||
        (st = dalloc(&h.leafmom, (long)kLeafMomStride * nleaf)) || (st = dalloc(&h.root, nc + kRootDoubles)) || (st = dalloc(&h.status, 1)) ||
        (st = dalloc(&h.site_ptr, 1)) ||
        (st = dalloc(&h.work, 8L * (depth >= 1 ? (1L << (3 * (depth - 1))) : 1) * ncp))) {
        free_all(h);
        delete H;
        return st;
    }
    h.epart_cap = (int)nleaf;
    if (!tiles.empty())
        cudaMemcpy(h.tiles, tiles.data(), sizeof(M2LTile) * tiles.size(), cudaMemcpyHostToDevice);
    if (!bricks.empty())
        cudaMemcpy(h.bricks, bricks.data(), sizeof(F32Brick) * bricks.size(), cudaMemcpyHostToDevice);
    cudaMemset(h.M, 0, sizeof(float) * acc * ncp);
    cudaMemset(h.L, 0, sizeof(float) * acc * ncp);
    cudaMemset(h.status, 0, sizeof(int));
    cudaMemset(h.leafcnt, 0, sizeof(uint32_t) * leafcnt_words(nleaf));
    cudaMemset(h.root, 0, sizeof(double) * (nc + kRootDoubles));
    cudaMemset(h.site_ptr, 0, sizeof(int));
    for (auto& e : h.ev) cudaEventCreate(&e);
    h.ev_valid = true;
    {
        int least = 0, greatest = 0;
        cudaDeviceGetStreamPriorityRange(&least, &greatest);
        if (cudaStreamCreateWithPriority(&h.chain, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaStreamCreateWithPriority(&h.side, cudaStreamNonBlocking, greatest) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h.gcap, cudaStreamNonBlocking) != cudaSuccess ||
            cudaStreamCreateWithFlags(&h.h2d, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.hx_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.hx_ev[1], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.hfree_ev[0], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.hfree_ev[1], cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.fork_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.eval_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.join_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.m2m_ev, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h.side_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            free_all(h);
            delete H;
            return FMM_ERR_CUDA;
        }
    }
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_all(h);
        delete H;
        return FMM_ERR_CUDA;
    }
    *out = H;
    return FMM_OK;
}

// Shared by fmm_set_charges (two forms per site, one lambda) and fmm_set_charges4 (four forms,
// two lambda coordinates per site, Sec. 2.1 Eq. 2).
static fmm_status set_charges_impl(fmm_handle* H, int n, int K, int nforms, const float* const* q,
                                   const int32_t* site, const float* lambda, void* stream) {
    if (!H || n < 0 || K < 0) return FMM_ERR_ARG;
    for (int f = 0; f < nforms; ++f)
        if (n > 0 && !q[f]) return FMM_ERR_ARG;
    if (n > 0 && !site) return FMM_ERR_ARG;
    if (K > 0 && !lambda) return FMM_ERR_ARG;
    Handle& h = H->h;
    cudaStream_t st = S(stream);
    const int ncoord = nforms == 4 ? 2 : 1;
    h.charges_set = false;
    if (n > h.cap || (nforms == 4 && !h.qC)) {
        free_atoms(h);
        fmm_status e;
        if ((e = dalloc(&h.qA, n)) || (e = dalloc(&h.qB, n)) || (e = dalloc(&h.site, n)) || (e = dalloc(&h.key, n)) ||
            (e = dalloc(&h.kA, n)) || (e = dalloc(&h.kB, n)) || (e = dalloc(&h.vA, n)) || (e = dalloc(&h.vB, n)) ||
            (e = dalloc(&h.inv, n)) || (e = dalloc(&h.pos, n)) || (e = dalloc(&h.dq, n)) ||
            (e = dalloc(&h.phis, n)) || (e = dalloc(&h.near, n)) || (e = dalloc(&h.near_items, n / 32 + 2)) ||
            (nforms == 4 && ((e = dalloc(&h.qC, n)) || (e = dalloc(&h.qD, n)) || (e = dalloc(&h.dqt, n))))) {
            free_atoms(h);
            return e;
        }
        h.cap = n;
        h.near_items_cap = n / 32 + 1;
        if ((e = cuda_ok(cudaMemset(h.near_items, 0, sizeof(int2))))) {
            free_atoms(h);
            return e;
        }
    }
    {  // one q phi partial per 128 atoms (k_far_out blocks)
        const int nparts = (n + 127) / 128;
        if (nparts > h.epart_cap) {
            dfree(h.epart);
            if (dalloc(&h.epart, nparts)) {
                h.epart_cap = 0;
                return FMM_ERR_OOM;
            }
            h.epart_cap = nparts;
        }
    }
    if (h.hamiltonian && (n > h.hi_cap || K > h.hi_kcap)) {
        dfree(h.hi_g);
        dfree(h.hi_site);
        h.hi_cap = h.hi_kcap = 0;
        if (dalloc(&h.hi_g, n > 0 ? n : 1) || dalloc(&h.hi_site, 3L * (K > 0 ? K : 1))) return FMM_ERR_OOM;
        h.hi_cap = n;
        h.hi_kcap = K;
    }
    if (ncoord * K > h.lam_cap) {
        dfree(h.lam);
        if (dalloc(&h.lam, ncoord * K)) return FMM_ERR_OOM;
        h.lam_cap = ncoord * K;
    }
    // site map: validated and grouped on the host (ascending input index within a site)
    std::vector<int32_t> hs(n);
    if (n > 0 && cudaMemcpyAsync(hs.data(), site, sizeof(int32_t) * n, cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return FMM_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return FMM_ERR_CUDA;
    std::vector<int> ptr(K + 1, 0);
    for (int i = 0; i < n; ++i) {
        if (hs[i] < -1 || hs[i] >= K) return FMM_ERR_ARG;
        if (hs[i] >= 0) ptr[hs[i] + 1]++;
    }
    for (int k = 0; k < K; ++k) ptr[k + 1] += ptr[k];
    std::vector<int> atoms(ptr[K] > 0 ? ptr[K] : 1);
    {
        std::vector<int> fill(ptr.begin(), ptr.end() - 1);
        for (int i = 0; i < n; ++i)
            if (hs[i] >= 0) atoms[fill[hs[i]]++] = i;
    }
    if (ptr[K] > h.site_cap || !h.site_atoms) {
        dfree(h.site_atoms);
        if (dalloc(&h.site_atoms, atoms.size())) return FMM_ERR_OOM;
        h.site_cap = (int)atoms.size();
    }
    dfree(h.site_ptr);
    if (dalloc(&h.site_ptr, ptr.size())) return FMM_ERR_OOM;
    fmm_status e = FMM_OK;
    if ((e = cuda_ok(cudaMemcpy(h.site_ptr, ptr.data(), sizeof(int) * ptr.size(), cudaMemcpyHostToDevice))) ||
        (e = cuda_ok(cudaMemcpy(h.site_atoms, atoms.data(), sizeof(int) * atoms.size(), cudaMemcpyHostToDevice))))
        return e;
    float* dst[4] = {h.qA, h.qB, h.qC, h.qD};
    if (n > 0) {
        for (int f = 0; f < nforms; ++f)
            if ((e = cuda_ok(cudaMemcpyAsync(dst[f], q[f], sizeof(float) * n, cudaMemcpyDeviceToDevice, st)))) return e;
        if ((e = cuda_ok(cudaMemcpyAsync(h.site, site, sizeof(int32_t) * n, cudaMemcpyDeviceToDevice, st)))) return e;
    }
    if (K > 0 &&
        (e = cuda_ok(cudaMemcpyAsync(h.lam, lambda, sizeof(float) * ncoord * K, cudaMemcpyDeviceToDevice, st))))
        return e;
    h.n = n;
    h.K = K;
    h.nforms = nforms;
    h.ncoord = ncoord;
    h.charges_set = true;
    ++h.gen;
    return FMM_OK;
}

fmm_status fmm_set_charges(fmm_handle* H, int n, int K, const float* qA, const float* qB, const int32_t* site,
                           const float* lambda, void* stream) {
    const float* q[2] = {qA, qB};
    return set_charges_impl(H, n, K, 2, q, site, lambda, stream);
}

fmm_status fmm_set_charges4(fmm_handle* H, int n, int K, const float* qA, const float* qB, const float* qC,
                            const float* qD, const int32_t* site, const float* lambda, void* stream) {
    const float* q[4] = {qA, qB, qC, qD};
    return set_charges_impl(H, n, K, 4, q, site, lambda, stream);
}

fmm_status fmm_set_lambda(fmm_handle* H, const float* lambda, void* stream) {
    if (!H) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.charges_set) return FMM_ERR_STATE;
    if (h.K == 0) return FMM_OK;
    if (!lambda) return FMM_ERR_ARG;
    return cuda_ok(cudaMemcpyAsync(h.lam, lambda, sizeof(float) * h.ncoord * h.K, cudaMemcpyDeviceToDevice, S(stream)));
}

fmm_status fmm_bind_lambda(fmm_handle* H, const float* lambda) {
    if (!H) return FMM_ERR_ARG;
    H->h.lam_bound = lambda;
    ++H->h.gen;
    return FMM_OK;
}

// One evaluation on `st`: a replay of one of the handle's two cached graphs when the buffers and
// the launch state are those it was captured with; captured (on the handle's own stream, into
// the least recently used slot) when the same buffers come again within the last two eager
// evaluations (so two buffer sets used in turn both get graphs); otherwise, while profiling, or
// while `st` is itself being captured by the caller, the kernels are launched one by one.  Both
// paths run the same kernels.
static fmm_status eval_launch(Handle& h, const float* x, double* E, float* F, float* dVdl, float* phi,
                              cudaStream_t st, bool capturing);

// An evaluation on a stream other than the last one's waits for the end of the last one's
// kernels (the handle's buffers are shared), but not for what that stream does after it, e.g.
// the copies of fmm_eval_host_async: a caller that alternates two streams overlaps one call's
// result copies with the next call's evaluation.  Inside the caller's own capture no cross-
// stream order is kept (the caller's graph orders its nodes).
static fmm_status eval_dispatch(Handle& h, const float* x, double* E, float* F, float* dVdl, float* phi,
                                cudaStream_t st) {
    cudaGetLastError();
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    cudaGetLastError();
    if (!capturing && h.eval_ev_valid && h.eval_last != st) {
        fmm_status e = cuda_ok(cudaStreamWaitEvent(st, h.eval_ev, 0));
        if (e) return e;
    }
    fmm_status e = eval_launch(h, x, E, F, dVdl, phi, st, capturing);
    if (e == FMM_OK && !capturing) {
        if ((e = cuda_ok(cudaEventRecord(h.eval_ev, st)))) return e;
        h.eval_last = st;
        h.eval_ev_valid = true;
    }
    return e;
}

static fmm_status eval_launch(Handle& h, const float* x, double* E, float* F, float* dVdl, float* phi,
                              cudaStream_t st, bool capturing) {
    const bool graphs = !h.profiling && !h.g_off && h.gcap && !capturing;
    if (graphs) {
        const void* key[5] = {x, E, F, dVdl, phi};
        auto same = [&](const void* const* k) {
            for (int i = 0; i < 5; ++i)
                if (k[i] != key[i]) return false;
            return true;
        };
        for (auto& g : h.g_slot)
            if (g.exec && g.gen == h.gen && same(g.key)) {
                g.used = ++h.g_tick;
                TraceRange trace("fmm:eval (graph)");
                return cuda_ok(cudaGraphLaunch(g.exec, st));
            }
        bool seen = false;
        for (int i = 0; i < 2; ++i) seen = seen || (h.g_hist_gen[i] == h.gen && same(h.g_hist[i]));
        if (seen) {
            Handle::EvalGraph& g = (!h.g_slot[0].exec || (h.g_slot[1].exec && h.g_slot[0].used <= h.g_slot[1].used))
                                       ? h.g_slot[0] : h.g_slot[1];
            if (g.exec) cudaGraphExecDestroy(g.exec);
            g.exec = nullptr;
            cudaGraph_t gr = nullptr;
            bool ok = cudaStreamBeginCapture(h.gcap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
            if (ok) {
                launch_eval(&h, x, E, F, dVdl, phi, h.gcap);
                ok = cudaStreamEndCapture(h.gcap, &gr) == cudaSuccess && gr != nullptr;
                // per-node priorities: the chain keeps the precedence its stream gives it eagerly
                ok = ok && cudaGraphInstantiateWithFlags(&g.exec, gr, cudaGraphInstantiateFlagUseNodePriority) ==
                               cudaSuccess;
                if (gr) cudaGraphDestroy(gr);
            }
            if (ok) {
                for (int i = 0; i < 5; ++i) g.key[i] = key[i];
                g.gen = h.gen;
                g.used = ++h.g_tick;
                return cuda_ok(cudaGraphLaunch(g.exec, st));
            }
            cudaGetLastError();  // capture is not available here: stay with eager launches
            for (auto& s2 : h.g_slot) {
                if (s2.exec) cudaGraphExecDestroy(s2.exec);
                s2.exec = nullptr;
            }
            h.g_off = true;
        } else {
            for (int i = 0; i < 5; ++i) h.g_hist[h.g_hist_next][i] = key[i];
            h.g_hist_gen[h.g_hist_next] = h.gen;
            h.g_hist_next ^= 1;
        }
    }
    launch_eval(&h, x, E, F, dVdl, phi, st);
    return cuda_ok(cudaGetLastError());
}

fmm_status fmm_stream_wait_eval(fmm_handle* H, void* stream) {
    if (!H) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.eval_ev_valid || h.eval_last == S(stream)) return FMM_OK;
    return cuda_ok(cudaStreamWaitEvent(S(stream), h.eval_ev, 0));
}

fmm_status fmm_eval(fmm_handle* H, const float* x, double* E, float* F, float* dVdl, float* phi, void* stream) {
    if (!H) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.charges_set) return FMM_ERR_STATE;
    if (h.n > 0 && !x) return FMM_ERR_ARG;
    return eval_dispatch(h, x, E, F, dVdl, phi, S(stream));
}

fmm_status fmm_eval_host_async(fmm_handle* H, const float* x_host, double* E_host, float* F_host, float* dV_host,
                               void* stream) {
    if (!H) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.charges_set) return FMM_ERR_STATE;
    if (h.n > 0 && !x_host) return FMM_ERR_ARG;
    cudaStream_t st = S(stream);
    const int n = h.n;
    const int nlam = h.ncoord * h.K;
    if (n > h.host_cap || !h.hE_dev[0] || nlam > h.hdV_cap) {
        // (re)allocate both staging sets; wait for any call still using them
        if (cudaDeviceSynchronize() != cudaSuccess) return cuda_fail("fmm_eval_host: synchronize", cudaGetLastError());
        h.host_cap = h.hdV_cap = 0;
        fmm_status e = FMM_OK;
        for (int i = 0; i < 2 && e == FMM_OK; ++i) {
            dfree(h.hx_dev[i]);
            dfree(h.hF_dev[i]);
            dfree(h.hE_dev[i]);
            dfree(h.hdV_dev[i]);
            if ((e = dalloc(&h.hx_dev[i], 3L * n)) || (e = dalloc(&h.hF_dev[i], 3L * n)) ||
                (e = dalloc(&h.hE_dev[i], 1)) || (e = dalloc(&h.hdV_dev[i], nlam)))
                break;
        }
        if (e != FMM_OK) return e;
        h.host_cap = n;
        h.hdV_cap = nlam;
    }
    const int s = h.h_next;
    h.h_next ^= 1;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    const bool capturing = cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone;
    cudaGetLastError();
    fmm_status e = FMM_OK;
    if (n > 0) {
        const size_t bytes = sizeof(float) * 3 * n;
        if (!capturing) {
            // the copy runs on the handle's copy stream once this staging set's previous use has
            // finished, beside whatever `st` is still doing; `st` waits for it
            if ((e = cuda_ok(cudaStreamWaitEvent(h.h2d, h.hfree_ev[s], 0))) ||
                (e = cuda_ok(cudaMemcpyAsync(h.hx_dev[s], x_host, bytes, cudaMemcpyHostToDevice, h.h2d))) ||
                (e = cuda_ok(cudaEventRecord(h.hx_ev[s], h.h2d))) || (e = cuda_ok(cudaStreamWaitEvent(st, h.hx_ev[s], 0))))
                return e;
        } else if ((e = cuda_ok(cudaMemcpyAsync(h.hx_dev[s], x_host, bytes, cudaMemcpyHostToDevice, st)))) {
            return e;
        }
    }
    if ((e = eval_dispatch(h, h.hx_dev[s], h.hE_dev[s], F_host ? h.hF_dev[s] : nullptr, dV_host ? h.hdV_dev[s] : nullptr,
                           nullptr, st)))
        return e;
    if (E_host && (e = cuda_ok(cudaMemcpyAsync(E_host, h.hE_dev[s], sizeof(double), cudaMemcpyDeviceToHost, st))))
        return e;
    if (F_host && n > 0 &&
        (e = cuda_ok(cudaMemcpyAsync(F_host, h.hF_dev[s], sizeof(float) * 3 * n, cudaMemcpyDeviceToHost, st))))
        return e;
    if (dV_host && nlam > 0 &&
        (e = cuda_ok(cudaMemcpyAsync(dV_host, h.hdV_dev[s], sizeof(float) * nlam, cudaMemcpyDeviceToHost, st))))
        return e;
    if (!capturing) e = cuda_ok(cudaEventRecord(h.hfree_ev[s], st));
    return e;
}

fmm_status fmm_eval_host(fmm_handle* H, const float* x_host, double* E_host, float* F_host, float* dV_host,
                         void* stream) {
    const fmm_status e = fmm_eval_host_async(H, x_host, E_host, F_host, dV_host, stream);
    if (e != FMM_OK) return e;
    return cuda_ok(cudaStreamSynchronize(S(stream)));
}

fmm_status fmm_host_alloc(size_t bytes, void** out) {
    if (!out) return FMM_ERR_ARG;
    *out = nullptr;
    if (bytes == 0) return FMM_ERR_ARG;
    if (cudaHostAlloc(out, bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        *out = nullptr;
        return FMM_ERR_OOM;
    }
    return FMM_OK;
}

void fmm_host_free(void* p) {
    if (p) cudaFreeHost(p);
}

fmm_status fmm_adjoint(fmm_handle* H, const double* gbar, const float* F, const float* phi, const float* dVdl,
                       float* gx, float* gqA, float* gqB, float* glam, void* stream) {
    if (!H || !gbar) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.charges_set) return FMM_ERR_STATE;
    if (gx && !F) return FMM_ERR_ARG;
    if ((gqA || gqB) && !phi) return FMM_ERR_ARG;
    if (glam && h.K > 0 && !dVdl) return FMM_ERR_ARG;
    if (h.nforms != 2) return FMM_ERR_STATE;  // four-form sites: fmm_adjoint4
    cudaGetLastError();
    float* gq[4] = {gqA, gqB, nullptr, nullptr};
    launch_adjoint(&h, gbar, F, phi, dVdl, gx, gq, glam, S(stream));
    return cuda_ok(cudaGetLastError());
}

fmm_status fmm_adjoint4(fmm_handle* H, const double* gbar, const float* F, const float* phi, const float* dVdl,
                        float* gx, float* gqA, float* gqB, float* gqC, float* gqD, float* glam, void* stream) {
    if (!H || !gbar) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.charges_set) return FMM_ERR_STATE;
    if (h.nforms != 4) return FMM_ERR_STATE;  // two-form sites: fmm_adjoint
    if (gx && !F) return FMM_ERR_ARG;
    if ((gqA || gqB || gqC || gqD) && !phi) return FMM_ERR_ARG;
    if (glam && h.K > 0 && !dVdl) return FMM_ERR_ARG;
    cudaGetLastError();
    float* gq[4] = {gqA, gqB, gqC, gqD};
    launch_adjoint(&h, gbar, F, phi, dVdl, gx, gq, glam, S(stream));
    return cuda_ok(cudaGetLastError());
}

fmm_status fmm_get_binning(fmm_handle* H, uint32_t* key, uint32_t* perm, uint32_t* start, uint32_t* count,
                           void* stream) {
    if (!H) return FMM_ERR_ARG;
    Handle& h = H->h;
    if (!h.charges_set || !h.perm) return FMM_ERR_STATE;
    cudaStream_t st = S(stream);
    const size_t nleaf = 1ul << (3 * h.depth);
    fmm_status e = FMM_OK;
    if (key && h.n && (e = cuda_ok(cudaMemcpyAsync(key, h.key, 4ul * h.n, cudaMemcpyDeviceToDevice, st)))) return e;
    if (perm && h.n && (e = cuda_ok(cudaMemcpyAsync(perm, h.perm, 4ul * h.n, cudaMemcpyDeviceToDevice, st))))
        return e;
    if (start && (e = cuda_ok(cudaMemcpyAsync(start, h.start, 4ul * nleaf, cudaMemcpyDeviceToDevice, st)))) return e;
    if (count && (e = cuda_ok(cudaMemcpyAsync(count, h.count, 4ul * nleaf, cudaMemcpyDeviceToDevice, st)))) return e;
    return FMM_OK;
}

fmm_status fmm_status_word(fmm_handle* H, int* device_status, void* stream) {
    if (!H || !device_status) return FMM_ERR_ARG;
    Handle& h = H->h;
    cudaStream_t st = S(stream);
    fmm_status e;
    if ((e = cuda_ok(cudaStreamSynchronize(st)))) return e;
    if ((e = cuda_ok(cudaMemcpy(device_status, h.status, sizeof(int), cudaMemcpyDeviceToHost)))) return e;
    // the bounds-checked build's index-check words (always 0 otherwise)
    const int bc[3] = {bc_take_kernels(), bc_take_m2l(), bc_take_translate()};
    const char* files[3] = {"kernels.cu", "m2l_tc.cu", "translate_tc.cu"};
    for (int i = 0; i < 3; ++i)
        if (bc[i]) {
            if (!(*device_status & FMM_DEV_BOUNDS))
                snprintf(g_last_error, sizeof(g_last_error), "index check failed at %s:%d", files[i], bc[i]);
            *device_status |= FMM_DEV_BOUNDS;
        }
    return cuda_ok(cudaMemset(h.status, 0, sizeof(int)));
}

int fmm_build_flags(void) {
#ifdef FMM_BOUNDS_CHECK
    return FMM_BUILD_BOUNDS_CHECK;
#else
    return 0;
#endif
}

fmm_status fmm_inject_alloc_failure(int n) {
    if (n < 0) return FMM_ERR_ARG;
    g_fail_alloc_in.store(n);
    return FMM_OK;
}

fmm_status fmm_inject_copy_loss(fmm_handle* H, int mask) {
    if (!H || (mask & ~(FMM_LOSE_TRANSLATE | FMM_LOSE_NEAR))) return FMM_ERR_ARG;
    H->h.copy_loss = mask;
    ++H->h.gen;  // a kernel argument: the captured evaluation graph no longer applies
    return FMM_OK;
}

fmm_status fmm_set_wait_limit(fmm_handle* H, long long cycles) {
    if (!H) return FMM_ERR_ARG;
    H->h.wait_limit = cycles > 0 ? cycles : 0;
    ++H->h.gen;  // a kernel argument: the captured evaluation graph no longer applies
    return FMM_OK;
}

fmm_status fmm_set_profiling(fmm_handle* H, int enable) {
    if (!H) return FMM_ERR_ARG;
    if (enable < 0 || enable > 2) return FMM_ERR_ARG;
    H->h.profiling = enable;
    ++H->h.gen;
    return FMM_OK;
}

int fmm_stage_times(fmm_handle* H, float* ms, int n) {
    if (!H || !ms || !H->h.profiling) return 0;
    Handle& h = H->h;
    if (h.ev_used <= 0 || cudaEventSynchronize(h.ev[h.ev_used - 1]) != cudaSuccess) {  // the last one recorded
        cudaGetLastError();
        return 0;
    }
    int k = 0;
    for (; k < n && k < kNumStages; ++k) {
        float t = 0.f;
        const int a = h.stage_ev[k][0], b = h.stage_ev[k][1];
        if (a >= 0 && b >= 0 && cudaEventElapsedTime(&t, h.ev[a], h.ev[b]) != cudaSuccess) {
            cudaGetLastError();
            t = -1.f;
        }
        ms[k] = t;
    }
    return k;
}

int fmm_launches_per_eval(const fmm_handle* H) { return H ? launches_per_eval(&H->h) : 0; }

void fmm_destroy(fmm_handle* H) {
    if (!H) return;
    cudaDeviceSynchronize();
    m2l_tc_free(&H->h);
    free_all(H->h);
    delete H;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Batches of independent replicas.  One fmm_batch_eval runs every replica's evaluation as a
// parallel branch of one CUDA graph (captured on first use, re-captured when the caller's
// pointers change), so uneven replicas share the GPU and the whole batch is one launch.
struct fmm_batch {
    std::vector<fmm_handle*> reps;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // [0] fork, [1..n] joins
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void*> key;     // pointers the graph was captured with
};

extern "C" {

fmm_status fmm_batch_create(int n, fmm_handle* const* handles, fmm_batch** out) {
    if (!out || n <= 0 || !handles) return FMM_ERR_ARG;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!handles[i]) return FMM_ERR_ARG;
    fmm_batch* b = new (std::nothrow) fmm_batch();
    if (!b) return FMM_ERR_OOM;
    b->reps.assign(handles, handles + n);
    b->streams.resize(n);
    b->events.resize(n + 1);
    for (int i = 0; i < n; ++i)
        if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            fmm_batch_destroy(b);
            return FMM_ERR_CUDA;
        }
    for (auto& e : b->events)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            fmm_batch_destroy(b);
            return FMM_ERR_CUDA;
        }
    *out = b;
    return FMM_OK;
}

fmm_status fmm_batch_eval(fmm_batch* b, const float* const* x, double* const* E, float* const* F,
                          float* const* dVdlambda, void* stream) {
    if (!b || !x || !E) return FMM_ERR_ARG;
    const int n = (int)b->reps.size();
    for (int i = 0; i < n; ++i) {
        if (!b->reps[i]->h.charges_set) return FMM_ERR_STATE;
        if (!E[i] || (b->reps[i]->h.n > 0 && !x[i])) return FMM_ERR_ARG;
    }
    std::vector<const void*> key;
    for (int i = 0; i < n; ++i) {
        key.push_back(x[i]);
        key.push_back(E[i]);
        key.push_back(F ? F[i] : nullptr);
        key.push_back(dVdlambda ? dVdlambda[i] : nullptr);
        key.push_back(b->reps[i]->h.lam_bound);
        key.push_back(b->reps[i]->h.perm);  // buffer growth re-captures
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaGetLastError();
    if (!b->exec || key != b->key) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        if (b->graph) cudaGraphDestroy(b->graph);
        b->exec = nullptr;
        b->graph = nullptr;
        // capture on a private stream: fork to one stream per replica, join back
        cudaStream_t origin = nullptr;
        cudaError_t ce = cudaStreamCreateWithFlags(&origin, cudaStreamNonBlocking);
        if (ce != cudaSuccess) return cuda_fail("fmm_batch_eval: stream", ce);
        fmm_status e = FMM_OK;
        ce = cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal);
        if (ce != cudaSuccess) e = cuda_fail("fmm_batch_eval: begin capture", ce);
        if (e == FMM_OK) {
            char where[96] = "";
            cudaError_t le = cudaEventRecord(b->events[0], origin);
            if (le != cudaSuccess) snprintf(where, sizeof(where), "fork record");
            for (int i = 0; i < n && le == cudaSuccess; ++i) {
                le = cudaStreamWaitEvent(b->streams[i], b->events[0], 0);
                if (le != cudaSuccess) { snprintf(where, sizeof(where), "fork wait, replica %d", i); break; }
                launch_eval(&b->reps[i]->h, x[i], E[i], F ? F[i] : nullptr, dVdlambda ? dVdlambda[i] : nullptr,
                            nullptr, b->streams[i]);
                le = cudaGetLastError();
                if (le != cudaSuccess) { snprintf(where, sizeof(where), "kernels of replica %d", i); break; }
                le = cudaEventRecord(b->events[i + 1], b->streams[i]);
                if (le != cudaSuccess) { snprintf(where, sizeof(where), "join record, replica %d", i); break; }
                le = cudaStreamWaitEvent(origin, b->events[i + 1], 0);
                if (le != cudaSuccess) { snprintf(where, sizeof(where), "join wait, replica %d", i); break; }
            }
            ce = cudaStreamEndCapture(origin, &b->graph);
            if (le != cudaSuccess) {
                char msg[160];
                snprintf(msg, sizeof(msg), "fmm_batch_eval: capture (%s)", where);
                e = cuda_fail(msg, le);
            } else if (ce != cudaSuccess) {
                e = cuda_fail("fmm_batch_eval: end capture", ce);
            }
        }
        if (e == FMM_OK) {
            ce = cudaGraphInstantiate(&b->exec, b->graph, 0);
            if (ce != cudaSuccess) e = cuda_fail("fmm_batch_eval: instantiate", ce);
        }
        cudaStreamDestroy(origin);
        if (e != FMM_OK) return e;
        b->key = key;
    }
    TraceRange trace("fmm:batch");  // the kernels of one batched evaluation, for a profiler
    const cudaError_t le = cudaGraphLaunch(b->exec, st);
    if (le != cudaSuccess) return cuda_fail("fmm_batch_eval: graph launch", le);
    return FMM_OK;
}

void fmm_batch_destroy(fmm_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    for (auto s : b->streams)
        if (s) cudaStreamDestroy(s);
    for (auto e : b->events)
        if (e) cudaEventDestroy(e);
    delete b;
}

}  // extern "C"
