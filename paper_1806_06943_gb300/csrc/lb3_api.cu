// lb3_api.cu -- C-ABI of the three-dimensional extension (declared in lb.h):
// parameter checks, device memory, stream ordering, host<->device transfers.
// All arithmetic of the method runs in the kernels of lb3_kernels.cuh.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lb.h"
#include "lb3_launch.h"
#include "lb_launch.h"

namespace {

int fail3(int code, const std::string &msg)
{
    lbk::set_last_error(msg.c_str());
    return code;
}

int cuda_fail3(cudaError_t e, const char *what)
{
    cudaGetLastError();
    return fail3(LB_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LB3_CUDA(call)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail3(e_, #call); \
    } while (0)

template <typename real>
void fill3(lbk3::Lat3<real> &L, const lb3_params &p)
{
    std::memset(&L, 0, sizeof L);
    L.nx = p.nx;
    L.ny = p.ny;
    L.nz = p.nz;
    L.pitch = (p.nx + 31) / 32 * 32;
    L.plane = (size_t)L.pitch * p.ny * p.nz;
    L.tiles_x = (p.nx + lbk3::TX - 1) / lbk3::TX;
    L.tiles_y = (p.ny + lbk3::TY - 1) / lbk3::TY;
    L.tiles_z = (p.nz + lbk3::TZ - 1) / lbk3::TZ;
    const double wcls[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    for (int k = 0; k < 2; ++k) {
        const double omega = 1.0 / p.tau[k];
        L.omega[k] = (real)omega;
        for (int c = 0; c < 3; ++c) L.aw[k][c] = (real)((1.0 - 0.5 * omega) * wcls[c]);
    }
    L.G1 = (real)p.G1;
    L.G2 = (real)p.G2;
    L.GAB = (real)p.G_AB;
    for (int a = 0; a < 3; ++a) L.g[a] = (real)p.g[a];
}

}  // namespace

struct lb3_handle {
    lb3_params p;
    int device = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    lbk3::Lat3<double> L64;
    lbk3::Lat3<float> L32;
    void *pool = nullptr;
    double *partials = nullptr, *obs = nullptr, *tmp = nullptr;
    size_t tmp_elems = 0;
    int n_tiles = 0;
    int parity = 0;
    int64_t t = 0;

    ~lb3_handle()
    {
        if (stream) cudaStreamSynchronize(stream);
        cudaFree(pool);
        cudaFree(partials);
        cudaFree(obs);
        cudaFree(tmp);
        if (stream && own_stream) cudaStreamDestroy(stream);
    }
    bool f64() const { return p.precision == LB_FP64; }
    size_t cells() const { return (size_t)p.nx * p.ny * p.nz; }
    int ensure_tmp(size_t elems)
    {
        if (elems <= tmp_elems) return LB_OK;
        if (tmp) {
            LB3_CUDA(cudaStreamSynchronize(stream));
            cudaFree(tmp);
            tmp = nullptr;
            tmp_elems = 0;
        }
        if (cudaMalloc((void **)&tmp, elems * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return fail3(LB_ENOMEM, "lb3: cudaMalloc of the transfer buffer failed");
        }
        tmp_elems = elems;
        return LB_OK;
    }
    cudaError_t density(int par)
    {
        return f64() ? lbk3::Launch3<double>::density(L64, par, stream) : lbk3::Launch3<float>::density(L32, par, stream);
    }
    cudaError_t collide(int par)
    {
        return f64() ? lbk3::Launch3<double>::collide(L64, par, stream) : lbk3::Launch3<float>::collide(L32, par, stream);
    }
    cudaError_t observe(double *part, double *rho, double *u)
    {
        return f64() ? lbk3::Launch3<double>::observe(L64, parity, part, rho, u, stream)
                     : lbk3::Launch3<float>::observe(L32, parity, part, rho, u, stream);
    }
};

extern "C" {

int lb3_create(const lb3_params *p, lb3_handle **out)
{
    if (!out) return fail3(LB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!p) return fail3(LB_EINVAL, "params is NULL");
    if (p->nx < 5 || p->ny < 5 || p->nz < 5) return fail3(LB_EINVAL, "lb3: nx, ny and nz must be >= 5");
    if ((long long)p->nx * p->ny * p->nz > (1ll << 31)) return fail3(LB_EINVAL, "lb3: lattice too large (nx*ny*nz > 2^31)");
    for (int k = 0; k < 2; ++k)
        if (!std::isfinite(p->tau[k]) || !(p->tau[k] > 0.5)) return fail3(LB_EINVAL, "lb3: tau must be finite and > 1/2");
    const double vals[] = {p->G_AB, p->G1, p->G2, p->g[0], p->g[1], p->g[2]};
    for (double v : vals)
        if (!std::isfinite(v)) return fail3(LB_EINVAL, "lb3: non-finite coupling or force");
    if (p->precision != LB_FP64 && p->precision != LB_FP32) return fail3(LB_EINVAL, "lb3: precision must be LB_FP64 or LB_FP32");
    lb3_handle *h = new (std::nothrow) lb3_handle();
    if (!h) return fail3(LB_ENOMEM, "host allocation failed");
    h->p = *p;
    auto bail = [&](int rc) {
        delete h;
        return rc;
    };
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail3(LB_ECUDA, "no CUDA device"));
    }
    if (p->stream) {
        h->stream = (cudaStream_t)p->stream;
    } else {
        if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail3(LB_ECUDA, "cudaStreamCreateWithFlags failed"));
        }
        h->own_stream = true;
    }
    fill3(h->L64, *p);
    fill3(h->L32, *p);
    const size_t rs = h->f64() ? 8 : 4, plane = h->L64.plane;
    const size_t fbytes = (38 * plane * rs + 255) / 256 * 256, rbytes = (2 * plane * rs + 255) / 256 * 256;
    const size_t total = 2 * fbytes + 2 * rbytes;
    h->n_tiles = h->L64.tiles_x * h->L64.tiles_y * h->L64.tiles_z;
    if (cudaMalloc(&h->pool, total) != cudaSuccess ||
        cudaMalloc((void **)&h->partials, (size_t)h->n_tiles * lbk3::kNumAcc * sizeof(double)) != cudaSuccess ||
        cudaMalloc((void **)&h->obs, lbk3::kNumAcc * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail3(LB_ENOMEM, "lb3: cudaMalloc of the lattice state failed"));
    }
    if (cudaMemsetAsync(h->pool, 0, total, h->stream) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail3(LB_ECUDA, "cudaMemsetAsync failed"));
    }
    char *b = (char *)h->pool;
    void *f0 = b, *f1 = b + fbytes, *r0 = b + 2 * fbytes, *r1 = b + 2 * fbytes + rbytes;
    h->L64.f[0] = (double *)f0;
    h->L64.f[1] = (double *)f1;
    h->L64.rho[0] = (double *)r0;
    h->L64.rho[1] = (double *)r1;
    h->L32.f[0] = (float *)f0;
    h->L32.f[1] = (float *)f1;
    h->L32.rho[0] = (float *)r0;
    h->L32.rho[1] = (float *)r1;
    *out = h;
    return LB_OK;
}

void lb3_destroy(lb3_handle *h) { delete h; }

#define CHECK3(h) \
    if (!(h)) return fail3(LB_EINVAL, "handle is NULL")

int lb3_set_fields(lb3_handle *h, const double *rho, const double *u)
{
    CHECK3(h);
    if (!rho) return fail3(LB_EINVAL, "rho is NULL");
    const size_t n = h->cells();
    int rc = h->ensure_tmp(5 * n);
    if (rc) return rc;
    LB3_CUDA(cudaMemcpyAsync(h->tmp, rho, 2 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    if (u) LB3_CUDA(cudaMemcpyAsync(h->tmp + 2 * n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, h->stream));
    h->parity = 0;
    h->t = 0;
    if (h->f64()) LB3_CUDA(lbk3::Launch3<double>::init(h->L64, h->tmp, u ? h->tmp + 2 * n : nullptr, 0, h->stream));
    else LB3_CUDA(lbk3::Launch3<float>::init(h->L32, h->tmp, u ? h->tmp + 2 * n : nullptr, 0, h->stream));
    LB3_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb3_step(lb3_handle *h, int64_t n)
{
    CHECK3(h);
    if (n < 0) return fail3(LB_EINVAL, "negative step count");
    for (int64_t s = 0; s < n; ++s) {
        LB3_CUDA(h->density(h->parity));
        LB3_CUDA(h->collide(h->parity));
        h->parity ^= 1;
        h->t += 1;
    }
    return LB_OK;
}

int64_t lb3_time(const lb3_handle *h) { return h ? h->t : -1; }

int lb3_set_probe(lb3_handle *h, double cx, double cy, double cz, double R)
{
    CHECK3(h);
    if (!std::isfinite(cx) || !std::isfinite(cy) || !std::isfinite(cz) || !std::isfinite(R))
        return fail3(LB_EINVAL, "non-finite probe");
    const double pr[4] = {cx, cy, cz, R};
    h->L64.has_probe = h->L32.has_probe = R > 0.0 ? 1 : 0;
    std::memcpy(h->L64.probe, pr, sizeof pr);
    std::memcpy(h->L32.probe, pr, sizeof pr);
    return LB_OK;
}

int lb3_observables(lb3_handle *h, lb3_obs *o)
{
    CHECK3(h);
    if (!o) return fail3(LB_EINVAL, "o is NULL");
    LB3_CUDA(h->density(h->parity));
    LB3_CUDA(h->observe(h->partials, nullptr, nullptr));
    LB3_CUDA(lbk3::reduce3(h->partials, h->n_tiles, h->obs, h->stream));
    double s[lbk3::kNumAcc];
    LB3_CUDA(cudaMemcpyAsync(s, h->obs, sizeof s, cudaMemcpyDeviceToHost, h->stream));
    LB3_CUDA(cudaStreamSynchronize(h->stream));
    std::memset(o, 0, sizeof *o);
    o->t = h->t;
    o->mass[0] = s[0];
    o->mass[1] = s[1];
    for (int a = 0; a < 3; ++a) {
        o->mom[0][a] = s[2 + a];
        o->mom[1][a] = s[5 + a];
    }
    o->umax = s[8];
    o->finite = s[9] == 0.0 ? 1 : 0;
    const double nan = std::nan("");
    if (h->L64.has_probe && s[12] > 0.0 && s[15] > 0.0) {
        const double rin = s[11] / s[12], rout = s[14] / s[15];
        o->dp_laplace = s[10] / s[12] - s[13] / s[15];
        o->R_eff = std::cbrt(3.0 * (s[0] - rout * (double)h->cells()) / (4.0 * 3.14159265358979323846 * (rin - rout)));
    } else {
        o->dp_laplace = nan;
        o->R_eff = nan;
    }
    if (!o->finite) return fail3(LB_EUNSTABLE, "a density or velocity is not finite");
    return LB_OK;
}

int lb3_get_fields(lb3_handle *h, double *rho, double *ubar)
{
    CHECK3(h);
    const size_t n = h->cells();
    int rc = h->ensure_tmp(5 * n);
    if (rc) return rc;
    LB3_CUDA(h->density(h->parity));
    LB3_CUDA(h->observe(nullptr, h->tmp, h->tmp + 2 * n));
    if (rho) LB3_CUDA(cudaMemcpyAsync(rho, h->tmp, 2 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    if (ubar) LB3_CUDA(cudaMemcpyAsync(ubar, h->tmp + 2 * n, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB3_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb3_get_populations(lb3_handle *h, double *f)
{
    CHECK3(h);
    if (!f) return fail3(LB_EINVAL, "f is NULL");
    const size_t n = h->cells();
    int rc = h->ensure_tmp(38 * n);
    if (rc) return rc;
    if (h->f64()) LB3_CUDA(lbk3::Launch3<double>::get_pops(h->L64, h->parity, h->tmp, h->stream));
    else LB3_CUDA(lbk3::Launch3<float>::get_pops(h->L32, h->parity, h->tmp, h->stream));
    LB3_CUDA(cudaMemcpyAsync(f, h->tmp, 38 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    LB3_CUDA(cudaStreamSynchronize(h->stream));
    return LB_OK;
}

int lb3_profile(lb3_handle *h, int32_t nsteps, void *flush_buf, size_t flush_bytes, double ms[3])
{
    CHECK3(h);
    if (nsteps < 1 || !ms) return fail3(LB_EINVAL, "profile needs nsteps >= 1 and ms");
    if (flush_bytes > 0 && !flush_buf) return fail3(LB_EINVAL, "flush_bytes > 0 with a NULL flush buffer");
    std::vector<cudaEvent_t> ev(3 * (size_t)nsteps, nullptr);
    auto cleanup = [&]() {
        for (auto &x : ev)
            if (x) cudaEventDestroy(x);
    };
    for (auto &x : ev)
        if (cudaEventCreate(&x) != cudaSuccess) {
            cleanup();
            cudaGetLastError();
            return fail3(LB_ECUDA, "cudaEventCreate failed");
        }
    cudaError_t ce = cudaSuccess;
    for (int s = 0; s < nsteps && ce == cudaSuccess; ++s) {
        if (flush_bytes) ce = cudaMemsetAsync(flush_buf, s & 0xff, flush_bytes, h->stream);
        if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s], h->stream);
        if (ce == cudaSuccess) ce = h->density(h->parity);
        if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s + 1], h->stream);
        if (ce == cudaSuccess) ce = h->collide(h->parity);
        if (ce == cudaSuccess) ce = cudaEventRecord(ev[3 * s + 2], h->stream);
        if (ce == cudaSuccess) {
            h->parity ^= 1;
            h->t += 1;
        }
    }
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int s = 0; s < nsteps && ce == cudaSuccess; ++s) {
        float a = 0.f, b = 0.f, c = 0.f;
        ce = cudaEventElapsedTime(&a, ev[3 * s], ev[3 * s + 1]);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&b, ev[3 * s + 1], ev[3 * s + 2]);
        if (ce == cudaSuccess) ce = cudaEventElapsedTime(&c, ev[3 * s], ev[3 * s + 2]);
        acc[0] += a;
        acc[1] += b;
        acc[2] += c;
    }
    cleanup();
    if (ce != cudaSuccess) return cuda_fail3(ce, "lb3 profiled time steps");
    for (int k = 0; k < 3; ++k) ms[k] = acc[k] / nsteps;
    return LB_OK;
}

}  // extern "C"
