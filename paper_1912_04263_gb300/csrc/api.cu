// C ABI of the gbosqp library (declared in include/gbosqp.h).  Every entry
// point validates its arguments, runs the C++ implementation, and turns any
// failure into a return code; no exception or abort crosses the boundary.
#include <chrono>
#include <mutex>
#include <cmath>
#include <memory>
#include <string>

#include "common.cuh"
#include "engine.cuh"
#include "handle.cuh"

namespace {

thread_local std::string g_setup_error;

int fail_code(gbosqp_handle *h, int code, const std::string &msg) {
    if (h) h->err = msg;
    return code;
}

#define API_TRY try {
#define API_CATCH(h)                                                                  \
    }                                                                                 \
    catch (const gb::GbError &e) { return fail_code(h, e.code, e.msg); }              \
    catch (const std::bad_alloc &) { return fail_code(h, GBOSQP_ERR_OOM, "host allocation failed"); } \
    catch (const std::exception &e) { return fail_code(h, GBOSQP_ERR_CUDA, e.what()); } \
    catch (...) { return fail_code(h, GBOSQP_ERR_CUDA, "unknown failure"); }

std::string check_settings(const gbosqp_settings &s) {
    if (!(s.alpha > 0.0 && s.alpha < 2.0)) return "alpha must be in ]0, 2[";
    if (!(s.sigma > 0.0) || !std::isfinite(s.sigma)) return "sigma must be > 0";
    if (!(s.rho0 > 0.0) || !std::isfinite(s.rho0)) return "rho0 must be > 0";
    if (!(s.eps_abs >= 0.0) || !(s.eps_rel >= 0.0)) return "eps_abs and eps_rel must be >= 0";
    if (!(s.pcg_lambda > 0.0 && s.pcg_lambda < 1.0)) return "pcg_lambda must be in ]0, 1[";
    if (!(s.pcg_eps_min > 0.0)) return "pcg_eps_min must be > 0";
    if (!(s.rho_min > 0.0) || !(s.rho_max >= s.rho_min)) return "need 0 < rho_min <= rho_max";
    if (!(s.eps_prim_inf >= 0.0) || !(s.eps_dual_inf >= 0.0) || !std::isfinite(s.eps_prim_inf) ||
        !std::isfinite(s.eps_dual_inf))
        return "eps_prim_inf and eps_dual_inf must be finite and >= 0";
    if (s.max_iter < 0 || s.max_cg_iter < 0) return "max_iter and max_cg_iter must be >= 0";
    if (s.check_every < 1 || s.check_every > 16) return "check_every must be in 1..16";
    if (s.rho_every < 0 || (s.rho_every > 0 && s.rho_every % s.check_every != 0))
        return "rho_every must be 0 or a multiple of check_every";
    if (s.scaling_iters < 0 || s.scaling_iters > 100) return "scaling_iters must be in 0..100";
    if (s.precision != GBOSQP_FP32 && s.precision != GBOSQP_FP64) return "precision must be FP32 or FP64";
    if (s.rho_policy < 0 || s.rho_policy > 2) return "unknown rho_policy";
    if (s.warm_start != 0 && s.warm_start != 1) return "warm_start must be 0 or 1";
    if (s.rho_vector != 0 && s.rho_vector != 1) return "rho_vector must be 0 or 1";
    if (s.pcg_variant != GBOSQP_PCG_CLASSIC && s.pcg_variant != GBOSQP_PCG_SINGLE_REDUCTION)
        return "pcg_variant must be GBOSQP_PCG_CLASSIC or GBOSQP_PCG_SINGLE_REDUCTION";
    if (s.rho_policy == GBOSQP_RHO_LEARNED && !s.policy_params) return "learned rho policy needs policy_params";
    if (s.input_location != GBOSQP_HOST && s.input_location != GBOSQP_DEVICE) return "bad input_location";
    if (s.loop_mode != GBOSQP_LOOP_GRAPH && s.loop_mode != GBOSQP_LOOP_HOST) return "bad loop_mode";
    return "";
}

int check_policy(const float *p) {
    // feature standard deviations and the clamp must be positive and finite
    for (int i = 0; i < GBOSQP_POLICY_PARAMS; ++i)
        if (!std::isfinite(p[i])) return GBOSQP_ERR_POLICY;
    for (int i = 4; i < 8; ++i)
        if (!(p[i] > 0.f)) return GBOSQP_ERR_POLICY;
    if (!(p[GBOSQP_POLICY_PARAMS - 4] > 0.f)) return GBOSQP_ERR_POLICY;
    return GBOSQP_OK;
}

}  // namespace

extern "C" {

int gbosqp_default_settings(gbosqp_settings *s) {
    if (!s) return GBOSQP_ERR_INVALID_ARG;
    *s = gbosqp_settings{};
    s->alpha = 1.6;
    s->sigma = 1e-6;
    s->rho0 = 0.1;
    s->eps_abs = 1e-3;
    s->eps_rel = 1e-3;
    s->pcg_lambda = 0.15;
    s->pcg_eps_min = 1e-7;
    s->rho_min = 1e-6;
    s->rho_max = 1e6;
    s->eps_prim_inf = 1e-4;
    s->eps_dual_inf = 1e-4;
    s->max_iter = 4000;
    s->max_cg_iter = 50;
    s->check_every = 5;
    s->rho_every = 10;
    s->scaling_iters = 10;
    s->precision = GBOSQP_FP32;
    s->rho_policy = GBOSQP_RHO_RATIO;
    s->P_is_upper = 1;
    s->input_location = GBOSQP_HOST;
    s->loop_mode = GBOSQP_LOOP_GRAPH;
    s->device = 0;
    s->warm_start = 0;
    s->rho_vector = 0;
    s->pcg_variant = GBOSQP_PCG_CLASSIC;
    s->cuda_stream = nullptr;
    s->policy_params = nullptr;
    return GBOSQP_OK;
}

const char *gbosqp_setup_error(void) { return g_setup_error.c_str(); }

int osqp_setup(gbosqp_handle **out, const gbosqp_csr *P, const gbosqp_csr *A, const double *q, const double *l,
               const double *u, const gbosqp_settings *settings) {
    g_setup_error.clear();
    if (!out) return GBOSQP_ERR_INVALID_ARG;
    *out = nullptr;
    auto bad = [](int code, const std::string &m) {
        g_setup_error = m;
        return code;
    };
    if (!P || !A || !q || !l || !u || !settings) return bad(GBOSQP_ERR_INVALID_ARG, "NULL argument");
    const gbosqp_settings &s = *settings;
    const std::string serr = check_settings(s);
    if (!serr.empty()) return bad(GBOSQP_ERR_INVALID_ARG, serr);
    if (s.rho_policy == GBOSQP_RHO_LEARNED && check_policy(s.policy_params) != GBOSQP_OK)
        return bad(GBOSQP_ERR_POLICY, "policy parameters are not finite or have a non-positive scale");
    const int n = P->nrows, m = A->nrows;
    if (n <= 0 || P->ncols != n) return bad(GBOSQP_ERR_DIMENSION, "P must be n x n with n > 0");
    if (m < 0 || A->ncols != n) return bad(GBOSQP_ERR_DIMENSION, "A must be m x n");
    if (P->nnz < 0 || A->nnz < 0) return bad(GBOSQP_ERR_CSR, "negative nnz");
    // offsets into the matrix arrays are 32-bit ints; 256 below 2^31 leaves room for the SpMV's
    // whole-batch loads past the last nonzero (up to 127 elements) and for offset arithmetic
    if (P->nnz >= (1LL << 31) - 256 || A->nnz >= (1LL << 31) - 256)
        return bad(GBOSQP_ERR_UNSUPPORTED, "2^31 - 256 or more nonzeros in one matrix");
    if (s.P_is_upper && 2 * P->nnz >= (1LL << 31) - 256)  // the full P has at most twice the upper triangle's entries
        return bad(GBOSQP_ERR_UNSUPPORTED,
                   "an upper-triangular P must have fewer than 2^30 - 128 nonzeros (its full form uses 32-bit offsets)");
    if ((int64_t)n + (int64_t)m >= (1LL << 31) - 256)
        return bad(GBOSQP_ERR_UNSUPPORTED, "n + m must be below 2^31 - 256 (the columns of [P A'] and the joint vectors)");
    if (!P->rowptr || (P->nnz && (!P->colind || !P->val)) || !A->rowptr || (A->nnz && (!A->colind || !A->val)))
        return bad(GBOSQP_ERR_INVALID_ARG, "NULL CSR array");
    std::unique_ptr<gbosqp_handle> h(new gbosqp_handle());
    h->s = s;
    try {
        GB_CUDA(cudaSetDevice(s.device));
        int cc_major = 0, cc_minor = 0;
        GB_CUDA(cudaDeviceGetAttribute(&cc_major, cudaDevAttrComputeCapabilityMajor, s.device));
        GB_CUDA(cudaDeviceGetAttribute(&cc_minor, cudaDevAttrComputeCapabilityMinor, s.device));
        if (cc_major * 10 + cc_minor != 103)
            gb::fail(GBOSQP_ERR_UNSUPPORTED, "device " + std::to_string(s.device) + " has compute capability " +
                                                 std::to_string(cc_major) + "." + std::to_string(cc_minor) +
                                                 ", not 10.3 (the library is compiled for sm_103a only)");
        if (s.cuda_stream) {
            h->stream = (cudaStream_t)s.cuda_stream;
        } else {
            GB_CUDA(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
            h->own_stream = true;
        }
        // device memory of the handle comes from the stream-ordered pool,
        // which keeps freed memory for reuse by later set-ups of this process
        static std::once_flag pool_once[64];
        if (s.device >= 0 && s.device < 64)
            std::call_once(pool_once[s.device], [&]() {
                cudaMemPool_t pool;
                if (cudaDeviceGetDefaultMemPool(&pool, s.device) == cudaSuccess) {
                    uint64_t keep = ~0ULL;
                    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
                }
                cudaGetLastError();
            });
        const auto t0 = std::chrono::steady_clock::now();
        const long long l0 = gb::g_launches;
        gb::PoolScope pool_scope(h->stream);
        // the SpMV plans are built on host threads while the device equilibrates
        std::shared_ptr<gb::PlanPrefetch> plans;
        gb::SetupData sd = gb::device_setup(*P, *A, q, l, u, s, h->stream,
                                            [&](std::vector<int> &&rpA, std::vector<int> &&rpP) {
                                                plans = gb::start_plans(s, std::move(rpA), std::move(rpP));
                                            });
        h->eng = gb::make_engine(std::move(sd), s, h->stream, std::move(plans));
        GB_CUDA(cudaStreamSynchronize(h->stream));
        h->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        h->setup_launches = gb::g_launches - l0;
    } catch (const gb::GbError &e) {
        g_setup_error = e.msg;
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        return e.code;
    } catch (const std::exception &e) {
        g_setup_error = e.what();
        if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
        return GBOSQP_ERR_CUDA;
    }
    *out = h.release();
    return GBOSQP_OK;
}

int osqp_solve(gbosqp_handle *h) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    const int st = h->eng->solve();
    h->eng->fill_info(h->info);
    return st;
    API_CATCH(h)
}

int osqp_update_rho(gbosqp_handle *h, double rho) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    if (!(rho > 0.0) || !std::isfinite(rho)) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "rho must be > 0 and finite");
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->update_rho(rho);
    return GBOSQP_OK;
    API_CATCH(h)
}

int osqp_warm_start(gbosqp_handle *h, const double *x, const double *y) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->warm_start(x, y);
    return GBOSQP_OK;
    API_CATCH(h)
}

int osqp_update_lin_cost(gbosqp_handle *h, const double *q) {
    if (!h || !h->eng || (!q && h->eng->n > 0)) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->update_lin_cost(q);
    return GBOSQP_OK;
    API_CATCH(h)
}

int osqp_update_bounds(gbosqp_handle *h, const double *l, const double *u) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->update_bounds(l, u);
    return GBOSQP_OK;
    API_CATCH(h)
}

int osqp_get_solution(const gbosqp_handle *hc, double *x, double *y, double *z) {
    gbosqp_handle *h = const_cast<gbosqp_handle *>(hc);
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->get_solution(x, y, z, false);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_get_solution_device(const gbosqp_handle *hc, double *x, double *y, double *z) {
    gbosqp_handle *h = const_cast<gbosqp_handle *>(hc);
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->get_solution(x, y, z, true);
    return GBOSQP_OK;
    API_CATCH(h)
}

int osqp_get_info(const gbosqp_handle *h, gbosqp_info *info) {
    if (!h || !info) return GBOSQP_ERR_INVALID_ARG;
    *info = h->info;
    info->setup_ms = h->setup_ms;
    info->setup_launches = h->setup_launches;
    if (h->eng) {
        info->nnz_A = h->eng->nnzA;
        info->nnz_P = h->eng->nnzP;
        info->solve_launches = h->eng->solve_launches;
    }
    return GBOSQP_OK;
}

void osqp_cleanup(gbosqp_handle *h) {
    if (!h) return;
    cudaSetDevice(h->s.device);
    if (h->stream) cudaStreamSynchronize(h->stream);
    h->eng.reset();
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
    delete h;
}

const char *gbosqp_last_error(const gbosqp_handle *h) { return h ? h->err.c_str() : "NULL handle"; }

const char *gbosqp_error_string(int code) {
    switch (code) {
        case GBOSQP_OK: return "ok";
        case GBOSQP_ERR_INVALID_ARG: return "invalid argument";
        case GBOSQP_ERR_DIMENSION: return "dimension mismatch";
        case GBOSQP_ERR_CSR: return "invalid CSR matrix";
        case GBOSQP_ERR_BOUNDS: return "invalid bounds (l > u or NaN)";
        case GBOSQP_ERR_NONFINITE: return "non-finite problem data";
        case GBOSQP_ERR_CUDA: return "CUDA error";
        case GBOSQP_ERR_OOM: return "out of device memory";
        case GBOSQP_ERR_DEVICE_TIMEOUT: return "device wait timed out";
        case GBOSQP_ERR_UNSUPPORTED: return "unsupported problem or device";
        case GBOSQP_ERR_POLICY: return "invalid learned-policy parameters";
        case GBOSQP_SOLVED: return "solved";
        case GBOSQP_MAX_ITER: return "maximum iterations reached";
        case GBOSQP_NONFINITE: return "non-finite iterates";
        case GBOSQP_PRIMAL_INFEASIBLE: return "primal infeasible";
        case GBOSQP_DUAL_INFEASIBLE: return "dual infeasible";
        default: return "unknown code";
    }
}

int gbosqp_dims(const gbosqp_handle *h, int32_t *n, int32_t *m, int64_t *nnz_A, int64_t *nnz_PAt) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    if (n) *n = h->eng->n;
    if (m) *m = h->eng->m;
    if (nnz_A) *nnz_A = h->eng->nnzA;
    if (nnz_PAt) *nnz_PAt = h->eng->nnzPAt;
    return GBOSQP_OK;
}

int gbosqp_get_scaling(const gbosqp_handle *hc, double *D, double *E, double *c) {
    gbosqp_handle *h = const_cast<gbosqp_handle *>(hc);
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->get_scaling(D, E, c);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_get_scaled_csr(const gbosqp_handle *hc, int which, int64_t *rowptr, int32_t *colind, double *val) {
    gbosqp_handle *h = const_cast<gbosqp_handle *>(hc);
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    if (which != GBOSQP_MAT_A && which != GBOSQP_MAT_PAT) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "bad matrix selector");
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->get_scaled_csr(which, rowptr, colind, val);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_spmv(gbosqp_handle *h, int which, const double *x, double *y, int fp64_accumulate) {
    if (!h || !h->eng || !x || !y) return GBOSQP_ERR_INVALID_ARG;
    if (which != GBOSQP_MAT_A && which != GBOSQP_MAT_PAT) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "bad matrix selector");
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->spmv(which, x, y, fp64_accumulate != 0);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_pcg(gbosqp_handle *h, double rho, const double *b, const double *x0, double eps, int32_t max_iter, double *x,
               int32_t *iters, double *r_norm) {
    if (!h || !h->eng || !b || !x0 || !x) return GBOSQP_ERR_INVALID_ARG;
    if (!(rho > 0.0) || !(eps >= 0.0) || max_iter < 0) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "bad rho, eps or max_iter");
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    int it = 0;
    double rn = 0.0;
    h->eng->pcg(rho, b, x0, eps, max_iter, x, &it, &rn);
    if (iters) *iters = it;
    if (r_norm) *r_norm = rn;
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_set_iterates(gbosqp_handle *h, const double *x, const double *z, const double *y, const double *xt,
                        double rho) {
    if (!h || !h->eng || !x || !z || !y || !xt) return GBOSQP_ERR_INVALID_ARG;
    if (!(rho > 0.0)) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "rho must be > 0");
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->set_iterates(x, z, y, xt, rho);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_get_iterates(const gbosqp_handle *hc, double *x, double *z, double *y, double *xt, double *rho) {
    gbosqp_handle *h = const_cast<gbosqp_handle *>(hc);
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->get_iterates(x, z, y, xt, rho);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_admm_iterations(gbosqp_handle *h, int32_t k, int32_t *pcg_per_iter) {
    if (!h || !h->eng || k < 0) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    const int st = h->eng->admm_iterations(k, pcg_per_iter);
    h->eng->fill_info(h->info);
    return st;
    API_CATCH(h)
}

int gbosqp_bench_kernel(gbosqp_handle *h, int kernel, int32_t reps, double *avg_ms) {
    if (!h || !h->eng || !avg_ms || reps < 0) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    *avg_ms = h->eng->bench_kernel(kernel, reps);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_resume(gbosqp_handle *h) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->resume();
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_set_pcg_lambda(gbosqp_handle *h, double lambda, double eps) {
    if (!h || !h->eng) return GBOSQP_ERR_INVALID_ARG;
    if (!(lambda > 0.0 && lambda < 1.0)) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "lambda must be in ]0, 1[");
    if (!(eps > 0.0) || !std::isfinite(eps)) return fail_code(h, GBOSQP_ERR_INVALID_ARG, "eps must be > 0");
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->set_lambda(lambda, eps);
    return GBOSQP_OK;
    API_CATCH(h)
}

int gbosqp_check(gbosqp_handle *h, double out[GBOSQP_CHECK_FIELDS]) {
    if (!h || !h->eng || !out) return GBOSQP_ERR_INVALID_ARG;
    API_TRY
    GB_CUDA(cudaSetDevice(h->s.device));
    h->eng->check(out);
    return GBOSQP_OK;
    API_CATCH(h)
}

}  // extern "C"
