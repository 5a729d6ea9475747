// Interfaces between device set-up (setup.cu), the per-precision solve
// engine (engine.cu) and the C ABI (api.cu).
#pragma once

#include <functional>
#include <memory>
#include <vector>

#include "common.cuh"

namespace gb {

// Output of device set-up: the equilibrated problem in FP64 on the device.
struct SetupData {
    int n = 0, m = 0;
    long long nnzA = 0, nnzPAt = 0, nnzP = 0;
    // A_bar (m x n) and [P_bar A_bar'] (n x (n+m)), CSR, int32 indices
    DevBuf A_rowptr, A_col, A_val;
    DevBuf PAt_rowptr, PAt_col, PAt_val, PAt_pend;
    std::vector<int> A_rowptr_host, PAt_rowptr_host;
    // vectors (double)
    DevBuf q, l, u, D, E, diagP, colsq;
    double c = 1.0;
    double qnorm_s = 0.0;  // ||q_bar||_inf
    double qnorm_u = 0.0;  // max_i |q_bar_i| / D_i  (times 1/c = ||q||_inf)
};

// Called by device_setup with the host row pointers of A and [P A'] as soon
// as they are known (before equilibration); the vectors are the callee's.
using RowptrHook = std::function<void(std::vector<int> &&A_rowptr, std::vector<int> &&PAt_rowptr)>;

// Build SetupData from validated inputs (see osqp_setup).  Throws GbError.
// With a hook, the host row pointers go to the hook instead of SetupData.
SetupData device_setup(const gbosqp_csr &P, const gbosqp_csr &A, const double *q, const double *l,
                       const double *u, const gbosqp_settings &s, cudaStream_t stream,
                       const RowptrHook &hook = RowptrHook());

// Host plans of the SpMV kernels, built on host threads from the row
// pointers while the device equilibrates, and handed to make_engine.
struct PlanPrefetch;
std::shared_ptr<PlanPrefetch> start_plans(const gbosqp_settings &s, std::vector<int> &&A_rowptr,
                                          std::vector<int> &&PAt_rowptr);

class EngineBase {
public:
    virtual ~EngineBase() = default;
    virtual int solve() = 0;                                   // returns status
    virtual void update_rho(double rho) = 0;
    virtual void warm_start(const double *x, const double *y) = 0;
    // parametric updates (scaled with the set-up's D, E, c); inputs on the
    // host or the device as settings.input_location says
    virtual void update_lin_cost(const double *q) = 0;
    virtual void update_bounds(const double *l, const double *u) = 0;
    virtual void get_solution(double *x, double *y, double *z, bool device) = 0;
    virtual void fill_info(gbosqp_info &info) = 0;
    virtual void get_scaling(double *D, double *E, double *c) = 0;
    virtual void get_scaled_csr(int which, int64_t *rowptr, int32_t *col, double *val) = 0;
    virtual void spmv(int which, const double *x, double *y, bool fp64acc) = 0;
    virtual void pcg(double rho, const double *b, const double *x0, double eps, int max_iter, double *x,
                     int *iters, double *rnorm) = 0;
    virtual void set_iterates(const double *x, const double *z, const double *y, const double *xt,
                              double rho) = 0;
    virtual void get_iterates(double *x, double *z, double *y, double *xt, double *rho) = 0;
    virtual int admm_iterations(int k, int *pcg_per_iter) = 0;
    virtual void check(double *out) = 0;
    virtual double bench_kernel(int kernel, int reps) = 0;
    virtual void set_lambda(double lambda, double eps) = 0;
    // the next solve continues from the current iterates, rho, PCG tolerance
    // and lambda (iteration count from 0)
    virtual void resume() = 0;
    // y = M x on device arrays of the working precision, with the split-row
    // scratch (tickets, partial sums) in the caller's device memory of
    // scratch_bytes bytes; allocates nothing.
    virtual void spmv_noalloc(int which, const void *x, void *y, unsigned char *scratch, size_t scratch_bytes) = 0;
    int n = 0, m = 0;
    long long solve_launches = 0;
    long long nnzA = 0, nnzPAt = 0, nnzP = 0;
};

std::unique_ptr<EngineBase> make_engine(SetupData &&sd, const gbosqp_settings &s, cudaStream_t stream,
                                        std::shared_ptr<PlanPrefetch> pre = nullptr);

}  // namespace gb
