// C ABI entry points (declared in include/lo_afqmc.h): argument checks,
// host/device buffer staging, workspace management and stage dispatch.
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>

using namespace loaf;

namespace {
void forget_plans(loaf_ctx* c);  // multi-system graphs using c
}  // namespace

namespace {

template <class F>
loaf_status guarded(loaf_ctx* c, F&& f) {
    try {
        f();
        if (c) c->err.clear();
        return LOAF_OK;
    } catch (const Error& e) {
        if (c) c->err = e.msg;
        return e.code;
    } catch (const std::exception& e) {
        if (c) c->err = e.what();
        return LOAF_ERR_CUDA;
    }
}

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // plain host memory on older drivers
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// per-walker status / logdet / energy from the per-spin parts
__global__ void finalize_kernel(int W, int nspin, double m0, double m1, double e0,
                                const double2* __restrict__ ld_part, const int* __restrict__ st_part,
                                const double2* __restrict__ e1, const double2* __restrict__ ej,
                                const double2* __restrict__ ek, double2* __restrict__ e_out,
                                double2* __restrict__ ld_out, int* __restrict__ st_out,
                                int* __restrict__ any_bad) {
    const int w = blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= W) return;
    int st = st_part[w];
    double2 ld = cscale(ld_part[w], m0 == 2.0 ? 2.0 : 1.0);
    if (nspin > 1) {
        st = max(st, st_part[W + w]);
        ld = cadd(ld, ld_part[W + w]);
    }
    (void)m1;
    double2 e = make_double2(e0, 0.0);
    if (e1) e = cadd(e, e1[w]);
    if (ej) e = cadd(e, ej[w]);
    if (ek) e = csub(e, ek[w]);
    if (st == LOAF_WALKER_OK && !(isfinite(e.x) && isfinite(e.y))) st = LOAF_WALKER_NAN;
    if (st != LOAF_WALKER_OK) {
        const double qnan = __longlong_as_double(0x7ff8000000000000LL);
        e = make_double2(qnan, qnan);
        atomicMax(any_bad, st);
    }
    if (e_out) e_out[w] = e;
    if (ld_out) ld_out[w] = ld;
    if (st_out) st_out[w] = st;
}

struct Staged {
    const double2* phi = nullptr;  // device copy of the walkers
};

// Workspace sized for W walkers (grown, never shrunk).
void ensure_workspace(loaf_ctx* c, int W, int mode) {
    const size_t wm = (size_t)W * c->ntot * c->M;
    c->w_phi.ensure(wm * sizeof(double2));
    c->w_theta.ensure(wm * sizeof(double2));
    c->w_z.ensure(wm * sizeof(double2));
    c->w_logdet.ensure((size_t)2 * W * sizeof(double2));
    c->w_status.ensure((size_t)2 * W * sizeof(int) + 16);
    c->w_out.ensure((size_t)3 * W * sizeof(double2));
    c->w_part2.ensure((size_t)W * (c->X + 1) * sizeof(double2));
    c->w_host_stage.ensure((size_t)W * (2 * sizeof(double2) + sizeof(int)) + 64);
    if (mode != LOAF_MODE_FULL) {
        long np = 0;
        for (int s = 0; s < c->nspin; ++s) np += c->sp[s].pairs.npairs;
        c->w_part.ensure((size_t)std::max<long>(np, 1) * W * sizeof(double2));
    }
    c->ws_W = std::max(c->ws_W, W);
}

const double2* stage_walkers(loaf_ctx* c, int W, const void* phi) {
    const size_t bytes = (size_t)W * c->M * c->ntot * sizeof(double2);
    if (is_device_ptr(phi)) return static_cast<const double2*>(phi);
    LOAF_CUDA(cudaMemcpyAsync(c->w_phi.ptr, phi, bytes, cudaMemcpyHostToDevice, c->stream));
    return c->w_phi.as<double2>();
}

// copy a device result to a user buffer that may live on the host
void deliver(loaf_ctx* c, void* user, const void* dev, size_t bytes) {
    if (!user) return;
    if (is_device_ptr(user)) {
        if (user != dev)
            LOAF_CUDA(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToDevice, c->stream));
    } else {
        LOAF_CUDA(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDeviceToHost, c->stream));
    }
}

void check_ready(loaf_ctx* c, int W, const void* phi, int mode, int precision) {
    LOAF_REQUIRE(c->loaded, LOAF_ERR_NOT_READY, "ao_load_cholesky has not been called");
    LOAF_REQUIRE(W >= 1, LOAF_ERR_ARG, "W must be >= 1");
    LOAF_REQUIRE(phi != nullptr, LOAF_ERR_ARG, "phi is NULL");
    LOAF_REQUIRE(mode == LOAF_MODE_FULL || mode == LOAF_MODE_LO || mode == LOAF_MODE_LO_JK, LOAF_ERR_ARG,
                 "unknown mode");
    LOAF_REQUIRE(mode != LOAF_MODE_LO_JK || c->closed, LOAF_ERR_UNSUPPORTED,
                 "the compressed Coulomb (LO_JK) is defined for closed shells");
    LOAF_REQUIRE(precision == LOAF_PREC_FP64 || precision == LOAF_PREC_FP16X3 ||
                     precision == LOAF_PREC_BF16X3 || precision == LOAF_PREC_FP16X3_F64INV ||
                     precision == LOAF_PREC_TF32,
                 LOAF_ERR_ARG, "unknown precision");
    LOAF_REQUIRE(precision != LOAF_PREC_TF32 || mode == LOAF_MODE_LO, LOAF_ERR_UNSUPPORTED,
                 "the TF32 precision is provided for the LO mode");
    LOAF_REQUIRE(mode == LOAF_MODE_FULL || c->compressed, LOAF_ERR_NOT_READY,
                 "LO mode needs lo_localize_compress");
}

// Theta for all walkers; returns 1 if any walker is singular or non-finite
void stage_theta(loaf_ctx* c, int W, const double2* phi) {
    run_theta_fp64(c, W, phi, c->w_theta.as<double2>(), c->w_logdet.as<double2>(),
                   c->w_status.as<int>());
}

}  // namespace

namespace loaf {

static cudaEvent_t prof_event(loaf_ctx* c) {
    if (!c->prof_pool.empty()) {
        cudaEvent_t e = c->prof_pool.back();
        c->prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    LOAF_CUDA(cudaEventCreate(&e));
    return e;
}

StageScope::StageScope(loaf_ctx* ctx, const char* name, int nlaunch) : c(ctx), launches(nlaunch) {
    if (!c->prof_on) return;
    for (size_t k = 0; k < c->prof.size(); ++k)
        if (c->prof[k].name == name) idx = (int)k;
    if (idx < 0) {
        c->prof.push_back(loaf_ctx::ProfStage{name});
        idx = (int)c->prof.size() - 1;
    }
    a = prof_event(c);
    b = prof_event(c);
    cudaEventRecord(a, c->stream);
}

void StageScope::end() {
    if (idx < 0) return;
    cudaEventRecord(b, c->stream);
    c->prof_open.push_back(loaf_ctx::ProfMark{idx, a, b, launches});
    idx = -1;
}

// wait for one submitted call and fold its flags into the context's
static void harvest_slot(loaf_ctx* c, loaf_ctx::AsyncSlot& s) {
    if (!s.pending) return;
    LOAF_CUDA(cudaEventSynchronize(s.done));
    c->async_flags[0] = std::max(c->async_flags[0], s.h_flags[0]);
    c->async_flags[1] |= s.h_flags[1];
    s.pending = false;
}

void drain_submitted(loaf_ctx* c) {
    const int a = c->aslot_next;  // the oldest call first
    harvest_slot(c, c->aslot[a]);
    harvest_slot(c, c->aslot[a ^ 1]);
}

void prof_collect(loaf_ctx* c) {
    for (auto& m : c->prof_open) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, m.a, m.b) == cudaSuccess) {
            c->prof[m.stage].total_ms += ms;
            c->prof[m.stage].calls += 1;
            c->prof[m.stage].launches += m.launches;
        }
        c->prof_pool.push_back(m.a);
        c->prof_pool.push_back(m.b);
    }
    c->prof_open.clear();
}

}  // namespace loaf

extern "C" {

loaf_status loaf_profile(loaf_ctx* c, int enable) {
    if (!c) return LOAF_ERR_ARG;
    return guarded(c, [&] {
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        prof_collect(c);
        c->prof.clear();
        c->prof_on = enable != 0;
    });
}

int loaf_profile_count(const loaf_ctx* c) { return c ? (int)c->prof.size() : 0; }

loaf_status loaf_test_withhold_stage(loaf_ctx* c, int n) {
    if (!c || n < 0) return LOAF_ERR_ARG;
    c->test_withhold = n;
    return LOAF_OK;
}

loaf_status loaf_set_tiles(loaf_ctx* c, int lo_chunk_cap, int coulomb_split) {
    if (!c) return LOAF_ERR_ARG;
    if (lo_chunk_cap < 64 || lo_chunk_cap > 256 || lo_chunk_cap % 32 != 0 || coulomb_split < 0 ||
        coulomb_split > 64) {
        c->err = "lo_chunk_cap must be a multiple of 32 in [64, 256] and coulomb_split in [0, 64]";
        return LOAF_ERR_ARG;
    }
    if (c->tile_lo_cap == lo_chunk_cap && c->tile_coul_split == coulomb_split) return LOAF_OK;
    return guarded(c, [&] {
        drain_submitted(c);
        c->tile_lo_cap = lo_chunk_cap;
        c->tile_coul_split = coulomb_split;
        c->tile_version += 1;
        forget_plans(c);
    });
}

loaf_status loaf_get_tiles(const loaf_ctx* c, int* lo_chunk_cap, int* coulomb_split) {
    if (!c) return LOAF_ERR_ARG;
    if (lo_chunk_cap) *lo_chunk_cap = c->tile_lo_cap;
    if (coulomb_split) *coulomb_split = c->tile_coul_split;
    return LOAF_OK;
}

loaf_status loaf_profile_get(const loaf_ctx* c, int idx, const char** name, double* total_ms,
                             long* calls, long* launches) {
    if (!c || idx < 0 || idx >= (int)c->prof.size()) return LOAF_ERR_ARG;
    if (name) *name = c->prof[idx].name.c_str();
    if (total_ms) *total_ms = c->prof[idx].total_ms;
    if (calls) *calls = c->prof[idx].calls;
    if (launches) *launches = c->prof[idx].launches;
    return LOAF_OK;
}


loaf_status loaf_create(loaf_ctx** out, int device, void* cuda_stream) {
    if (!out) return LOAF_ERR_ARG;
    *out = nullptr;
    loaf_ctx* c = new (std::nothrow) loaf_ctx();
    if (!c) return LOAF_ERR_OOM;
    loaf_status st = guarded(c, [&] {
        int n = 0;
        LOAF_CUDA(cudaGetDeviceCount(&n));
        LOAF_REQUIRE(device >= 0 && device < n, LOAF_ERR_ARG, "no such CUDA device");
        c->device = device;
        LOAF_CUDA(cudaSetDevice(device));
        LOAF_CUDA(cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device));
        if (cuda_stream) {
            c->stream = static_cast<cudaStream_t>(cuda_stream);
        } else {
            LOAF_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
            c->own_stream = true;
        }
        LOAF_CUBLAS(cublasCreate(&c->cublas));
        LOAF_CUBLAS(cublasSetStream(c->cublas, c->stream));
        LOAF_CUSOLVER(cusolverDnCreate(&c->cusolver));
        LOAF_CUSOLVER(cusolverDnSetStream(c->cusolver, c->stream));
    });
    if (st != LOAF_OK) {
        loaf_destroy(c);
        return st;
    }
    *out = c;
    return LOAF_OK;
}

loaf_status loaf_destroy(loaf_ctx* c) {
    if (!c) return LOAF_OK;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    forget_plans(c);
    if (c->branch_stream) cudaStreamDestroy(c->branch_stream);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->h_flags) cudaFreeHost(c->h_flags);
    for (auto& sl : c->aslot) {
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.h_flags) cudaFreeHost(sl.h_flags);
        sl.phi.release();
        sl.out.release();
    }
    for (auto& s : c->sp) s.release();
    for (auto& m : c->mix) m.release();
    c->d_h.release(); c->d_L.release();
    for (loaf::DevBuf* b : {&c->w_phi, &c->w_theta, &c->w_z, &c->w_lu, &c->w_perm, &c->w_logdet,
                            &c->w_status, &c->w_out, &c->w_part, &c->w_part2, &c->w_dhi,
                            &c->w_dlo, &c->w_dscale, &c->w_host_stage, &c->w_cpart,
                            &c->w_lopart, &c->w_red, &c->w_flag, &c->d_keep, &c->w_oz_at,
                            &c->w_oz_bt, &c->w_oz_S, &c->w_oz_int, &c->w_oz_key, &c->w_prop_x, &c->w_prop_part,
                            &c->w_dfull, &c->w_dtf})
        b->release();
    for (cudaStream_t cs : c->copy_stream)
        if (cs) cudaStreamDestroy(cs);
    for (cudaEvent_t e : {c->ev_start, c->ev_copied[0][0], c->ev_copied[0][1], c->ev_copied[1][0],
                          c->ev_copied[1][1], c->ev_free[0], c->ev_free[1]})
        if (e) cudaEventDestroy(e);
    if (c->cublas) cublasDestroy(c->cublas);
    if (c->cusolver) cusolverDnDestroy(c->cusolver);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
    return LOAF_OK;
}

const char* loaf_status_str(loaf_status s) {
    switch (s) {
        case LOAF_OK: return "ok";
        case LOAF_ERR_ARG: return "invalid argument";
        case LOAF_ERR_SHAPE: return "invalid or unsupported shape";
        case LOAF_ERR_CUDA: return "CUDA error";
        case LOAF_ERR_OOM: return "out of device memory";
        case LOAF_ERR_SINGULAR: return "singular walker overlap";
        case LOAF_ERR_NOT_READY: return "setup call missing";
        case LOAF_ERR_TIMEOUT: return "bounded device wait gave up";
        case LOAF_ERR_NAN: return "non-finite value";
        case LOAF_ERR_UNSUPPORTED: return "unsupported request";
    }
    return "unknown status";
}

const char* loaf_last_error(const loaf_ctx* c) { return c ? c->err.c_str() : "null context"; }

loaf_status ao_load_cholesky(loaf_ctx* c, int M, int X, const double* h, const double* L,
                             int n_alpha, int n_beta, const double* trial_a,
                             const double* trial_b, double e0, int inputs_on_device) {
    if (!c) return LOAF_ERR_ARG;
    return guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        drain_submitted(c);
        setup_load(c, M, X, h, L, n_alpha, n_beta, trial_a, trial_b, e0, inputs_on_device);
    });
}

loaf_status lo_localize_compress(loaf_ctx* c, double t_svd, const double* r_ops, int n_ops,
                                 int localize, double* compression_pct, int* m_svd_per_pair) {
    if (!c) return LOAF_ERR_ARG;
    return guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        drain_submitted(c);
        setup_compress(c, t_svd, r_ops, n_ops, localize, compression_pct, m_svd_per_pair);
    });
}

int loaf_num_pairs(const loaf_ctx* c) {
    if (!c || !c->compressed) return 0;
    int n = 0;
    for (int s = 0; s < c->nspin; ++s) n += c->sp[s].pairs.npairs;
    return n;
}

loaf_status lo_get_localized_trial(const loaf_ctx* c, int spin, double* out) {
    if (!c || !out) return LOAF_ERR_ARG;
    if (!c->loaded) return LOAF_ERR_NOT_READY;
    if (spin < 0 || spin >= c->nspin) return LOAF_ERR_ARG;
    std::memcpy(out, c->sp[spin].h_trial.data(), c->sp[spin].h_trial.size() * sizeof(double));
    return LOAF_OK;
}

loaf_status walkers_theta(loaf_ctx* c, int W, const void* phi, void* theta_out, void* logdet_out,
                          int* walker_status) {
    if (!c) return LOAF_ERR_ARG;
    int bad = 0;
    loaf_status st = guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        check_ready(c, W, phi, LOAF_MODE_FULL, LOAF_PREC_FP64);
        ensure_workspace(c, W, LOAF_MODE_FULL);
        const double2* dphi = stage_walkers(c, W, phi);
        stage_theta(c, W, dphi);
        double2* dld = c->w_host_stage.as<double2>();
        int* dst = reinterpret_cast<int*>(dld + W);
        int* dbad = dst + W;
        LOAF_CUDA(cudaMemsetAsync(dbad, 0, sizeof(int), c->stream));
        finalize_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
            W, c->nspin, c->sp[0].mult, c->nspin > 1 ? c->sp[1].mult : 0.0, 0.0,
            c->w_logdet.as<double2>(), c->w_status.as<int>(), nullptr, nullptr, nullptr, nullptr,
            dld, dst, dbad);
        LOAF_LAUNCH_CHECK();
        deliver(c, theta_out, c->w_theta.ptr, (size_t)W * c->ntot * c->M * sizeof(double2));
        deliver(c, logdet_out, dld, (size_t)W * sizeof(double2));
        deliver(c, walker_status, dst, (size_t)W * sizeof(int));
        LOAF_CUDA(cudaMemcpyAsync(&bad, dbad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
    });
    if (st == LOAF_OK && bad) {
        c->err = "at least one walker overlap is singular or non-finite";
        return bad == LOAF_WALKER_SINGULAR ? LOAF_ERR_SINGULAR : LOAF_ERR_NAN;
    }
    return st;
}

namespace {

__global__ void flag_or_kernel(const int* __restrict__ flag, int* __restrict__ acc) {
    if (*flag) *acc = 1;
}

// Theta, the energy terms and finalize for W walkers at dphi; the results go
// to de / dld / dst (device), the worst walker status to *dbad and any
// pipeline timeout to *dtimeout.
void energy_batch(loaf_ctx* c, int W, const double2* dphi, int mode, int precision, double2* de,
                  double2* dld, int* dst, int* dbad, int* dtimeout) {
    // the LO split-precision path forms Delta on the tensor cores; the FP64
    // path and the full mode use the FP64 Theta kernel
    const bool tc_theta = precision != LOAF_PREC_FP64 && mode != LOAF_MODE_FULL;
    if (tc_theta) {
        // the LO operands first: the dense blocks need an FP32 copy of Delta
        run_theta_tc(c, W, dphi, precision, prepare_lo_operands(c, mode, precision));
    } else {
        StageScope sc(c, "theta_fp64", c->nspin);
        stage_theta(c, W, dphi);
    }
    double2* e1 = c->w_out.as<double2>();
    double2* ej = e1 + W;
    double2* ek = ej + W;
    if (precision == LOAF_PREC_FP64) {
        {
            StageScope sc(c, "coulomb_fp64", 2);
            run_coulomb_fp64(c, W, c->w_theta.as<double2>(), e1);
        }
        if (mode == LOAF_MODE_FULL) {
            StageScope sc(c, "exchange_full_fp64", c->nspin + 1);
            run_energy_fp64_full(c, W, c->w_theta.as<double2>(), ek);
        } else {
            StageScope sc(c, "exchange_lo_fp64", 2 * c->nspin);
            run_energy_fp64_lo(c, W, c->w_theta.as<double2>(), ek, c->w_part.as<double2>());
        }
        if (mode == LOAF_MODE_LO_JK) {
            StageScope sc(c, "coulomb_lo_fp64", 2);
            run_coulomb_lo_fp64(c, W, c->w_theta.as<double2>(), ej, c->w_part.as<double2>());
        }
    } else {
        run_energy_mixed(c, W, mode, precision, tc_theta ? nullptr : c->w_theta.as<double2>(),
                         e1, nullptr);
    }
    StageScope fsc(c, "finalize_d2h", precision != LOAF_PREC_FP64 ? 2 : 1);
    finalize_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
        W, c->nspin, c->sp[0].mult, c->nspin > 1 ? c->sp[1].mult : 0.0, c->e0,
        c->w_logdet.as<double2>(), c->w_status.as<int>(), e1, ej, ek, de, dld, dst, dbad);
    LOAF_LAUNCH_CHECK();
    if (precision != LOAF_PREC_FP64) {
        flag_or_kernel<<<1, 1, 0, c->stream>>>(c->w_flag.as<int>(), dtimeout);
        LOAF_LAUNCH_CHECK();
    }
}

// the two upload streams and their events, created on first use
void ensure_copy_streams(loaf_ctx* c) {
    if (c->copy_stream[0]) return;
    for (cudaStream_t* cs : {&c->copy_stream[0], &c->copy_stream[1]})
        LOAF_CUDA(cudaStreamCreateWithFlags(cs, cudaStreamNonBlocking));
    for (cudaEvent_t* e : {&c->ev_start, &c->ev_copied[0][0], &c->ev_copied[0][1], &c->ev_copied[1][0],
                           &c->ev_copied[1][1], &c->ev_free[0], &c->ev_free[1]})
        LOAF_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
}

// Upload chunks for a host array of W walkers (empty: one piece).  At
// pentacene scale uploading a walker over the host link takes a little longer
// than computing it (about 10.3 against 8.8 us), so the copies run back to back
// and a call costs all the copies plus the compute of the last chunk: the
// chunks are 128 walkers (computing starts early), then 256, and the last one
// 128 again, each uploaded while the previous one computes.  Even and odd
// chunks alternate between two device buffers of at most 256 walkers each.
// Walkers per pass over the pipeline: larger batches run slower per walker at
// pentacene scale (65.5k walker energies/s at 1024, 60k at 2048 and 4096 on
// B300), so bigger calls are processed in slices of this size.
constexpr int kMaxBatch = 1024;

std::vector<int> host_chunks(int W) {
    std::vector<int> v;
    if (W < 512) return v;
    v.push_back(128);
    int rem = W - 128;
    while (rem - 256 >= 128) {
        v.push_back(256);
        rem -= 256;
    }
    if (rem > 256) {  // 257 .. 383 left: split so that the last chunk is 128
        v.push_back(rem - 128);
        rem = 128;
    }
    v.push_back(rem);
    return v;
}

}  // namespace

loaf_status walkers_energy(loaf_ctx* c, int W, const void* phi, int mode, int precision,
                           void* e_out, void* logdet_out, int* walker_status) {
    if (!c) return LOAF_ERR_ARG;
    int flags[2] = {0, 0};  // worst walker status, timeout
    loaf_status st = guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        check_ready(c, W, phi, mode, precision);
        LOAF_REQUIRE(e_out != nullptr, LOAF_ERR_ARG, "e_out is NULL");
        ensure_workspace(c, W, mode);
        double2* de = c->w_host_stage.as<double2>();
        double2* dld = de + W;
        int* dst = reinterpret_cast<int*>(dld + W);
        int* dflags = dst + W;  // [worst status, timeout]
        LOAF_CUDA(cudaMemsetAsync(dflags, 0, 2 * sizeof(int), c->stream));
        const std::vector<int> chunks = is_device_ptr(phi) ? std::vector<int>{} : host_chunks(W);
        if (chunks.empty()) {
            const double2* dphi;
            {
                StageScope sc(c, "h2d_walkers", 0);
                dphi = stage_walkers(c, W, phi);
            }
            const size_t per_w = (size_t)c->M * c->ntot;
            for (int w0 = 0; w0 < W; w0 += kMaxBatch) {
                const int Wk = std::min(kMaxBatch, W - w0);
                energy_batch(c, Wk, dphi + (size_t)w0 * per_w, mode, precision, de + w0, dld + w0, dst + w0,
                             dflags, dflags + 1);
            }
        } else {
            // upload chunk k + 1 on the copy stream while chunk k computes
            ensure_copy_streams(c);
            const size_t per_w = (size_t)c->M * c->ntot;
            const double2* hphi = static_cast<const double2*>(phi);
            int even_max = 0;
            for (size_t k = 0; k < chunks.size(); k += 2) even_max = std::max(even_max, chunks[k]);
            double2* buf[2] = {c->w_phi.as<double2>(), c->w_phi.as<double2>() + (size_t)even_max * per_w};
            LOAF_CUDA(cudaEventRecord(c->ev_start, c->stream));  // earlier users of w_phi are done
            for (cudaStream_t cs : c->copy_stream) LOAF_CUDA(cudaStreamWaitEvent(cs, c->ev_start, 0));
            int w0 = 0;
            for (size_t k = 0; k < chunks.size(); ++k) {
                const int b = (int)(k & 1), Wk = chunks[k];
                // the chunk's first and second halves of walkers on the two copy streams
                for (int h = 0; h < 2; ++h) {
                    const int a0 = h == 0 ? 0 : Wk / 2, a1 = h == 0 ? Wk / 2 : Wk;
                    cudaStream_t cs = c->copy_stream[h];
                    if (k >= 2) LOAF_CUDA(cudaStreamWaitEvent(cs, c->ev_free[b], 0));
                    LOAF_CUDA(cudaMemcpyAsync(buf[b] + (size_t)a0 * per_w, hphi + (size_t)(w0 + a0) * per_w,
                                              (size_t)(a1 - a0) * per_w * sizeof(double2), cudaMemcpyHostToDevice,
                                              cs));
                    LOAF_CUDA(cudaEventRecord(c->ev_copied[b][h], cs));
                    LOAF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_copied[b][h], 0));
                }
                energy_batch(c, Wk, buf[b], mode, precision, de + w0, dld + w0, dst + w0, dflags,
                             dflags + 1);
                LOAF_CUDA(cudaEventRecord(c->ev_free[b], c->stream));
                w0 += Wk;
            }
        }
        deliver(c, e_out, de, (size_t)W * sizeof(double2));
        deliver(c, logdet_out, dld, (size_t)W * sizeof(double2));
        deliver(c, walker_status, dst, (size_t)W * sizeof(int));
        LOAF_CUDA(cudaMemcpyAsync(flags, dflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        prof_collect(c);
    });
    if (st == LOAF_OK && flags[1]) {
        c->err = "a tensor-core kernel gave up waiting on a pipeline barrier";
        return LOAF_ERR_TIMEOUT;
    }
    if (st == LOAF_OK && flags[0]) {
        c->err = "at least one walker overlap is singular or non-finite";
        return flags[0] == LOAF_WALKER_SINGULAR ? LOAF_ERR_SINGULAR : LOAF_ERR_NAN;
    }
    return st;
}

// ---------------------------------------------------------------------------
// submitted calls: the upload of one call overlaps the compute of the previous
// ---------------------------------------------------------------------------
namespace {

constexpr int kUploadPieces = 16;

}  // namespace

loaf_status walkers_energy_submit(loaf_ctx* c, int W, const void* phi, int mode, int precision,
                                  void* e_out, void* logdet_out, int* walker_status) {
    if (!c) return LOAF_ERR_ARG;
    return guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        check_ready(c, W, phi, mode, precision);
        LOAF_REQUIRE(e_out != nullptr, LOAF_ERR_ARG, "e_out is NULL");
        // the workspace is sized for one (W, mode, precision); a call with
        // another first lets the calls in flight finish, so that no buffer
        // they use is reallocated under them
        const long long key = ((long long)W * 8 + mode) * 8 + precision;
        if (key != c->async_key) {
            drain_submitted(c);
            c->async_key = key;
        }
        loaf_ctx::AsyncSlot& sl = c->aslot[c->aslot_next];
        // only the call two back, which used this slot's buffers: the previous
        // call keeps computing while this one uploads
        harvest_slot(c, sl);
        if (!sl.done) {
            LOAF_CUDA(cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming));
            LOAF_CUDA(cudaMallocHost(&sl.h_flags, 2 * sizeof(int)));
        }
        ensure_workspace(c, W, mode);
        const size_t per_w = (size_t)c->M * c->ntot;
        sl.out.ensure((size_t)W * (2 * sizeof(double2) + sizeof(int)) + 64);
        double2* de = sl.out.as<double2>();
        double2* dld = de + W;
        int* dst = reinterpret_cast<int*>(dld + W);
        int* dflags = dst + W;
        LOAF_CUDA(cudaMemsetAsync(dflags, 0, 2 * sizeof(int), c->stream));
        const double2* dphi = static_cast<const double2*>(phi);
        if (!is_device_ptr(phi)) {
            // the whole call in up to 16 pieces taken in turn by the two copy
            // streams (52.5 GB/s over the host link as two halves, 55.4 as 16
            // pieces, measured on B300); they wait for nothing on the compute
            // stream (this slot's last call is done)
            ensure_copy_streams(c);
            sl.phi.ensure((size_t)W * per_w * sizeof(double2));
            const double2* hphi = static_cast<const double2*>(phi);
            double2* buf = sl.phi.as<double2>();
            const int pieces = std::min(W, kUploadPieces);
            for (int i = 0; i < pieces; ++i) {
                const int a0 = (int)((long)i * W / pieces), a1 = (int)((long)(i + 1) * W / pieces);
                LOAF_CUDA(cudaMemcpyAsync(buf + (size_t)a0 * per_w, hphi + (size_t)a0 * per_w,
                                          (size_t)(a1 - a0) * per_w * sizeof(double2), cudaMemcpyHostToDevice,
                                          c->copy_stream[i & 1]));
            }
            for (int h = 0; h < std::min(pieces, 2); ++h) {
                LOAF_CUDA(cudaEventRecord(c->ev_copied[0][h], c->copy_stream[h]));
                LOAF_CUDA(cudaStreamWaitEvent(c->stream, c->ev_copied[0][h], 0));
            }
            dphi = buf;
        }
        for (int w0 = 0; w0 < W; w0 += kMaxBatch) {
            const int Wk = std::min(kMaxBatch, W - w0);
            energy_batch(c, Wk, dphi + (size_t)w0 * per_w, mode, precision, de + w0, dld + w0, dst + w0,
                         dflags, dflags + 1);
        }
        deliver(c, e_out, de, (size_t)W * sizeof(double2));
        deliver(c, logdet_out, dld, (size_t)W * sizeof(double2));
        deliver(c, walker_status, dst, (size_t)W * sizeof(int));
        LOAF_CUDA(cudaMemcpyAsync(sl.h_flags, dflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaEventRecord(sl.done, c->stream));
        sl.pending = true;
        c->aslot_next ^= 1;
    });
}

loaf_status walkers_energy_wait(loaf_ctx* c) {
    if (!c) return LOAF_ERR_ARG;
    loaf_status st = guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        drain_submitted(c);
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        prof_collect(c);
    });
    const int worst = c->async_flags[0], timeout = c->async_flags[1];
    c->async_flags[0] = c->async_flags[1] = 0;
    if (st != LOAF_OK) return st;
    if (timeout) {
        c->err = "a tensor-core kernel gave up waiting on a pipeline barrier";
        return LOAF_ERR_TIMEOUT;
    }
    if (worst) {
        c->err = "at least one walker overlap is singular or non-finite";
        return worst == LOAF_WALKER_SINGULAR ? LOAF_ERR_SINGULAR : LOAF_ERR_NAN;
    }
    return LOAF_OK;
}

// ---------------------------------------------------------------------------
// several systems in one graph
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct MultiPlan {
    std::vector<loaf_ctx*> ctxs;
    std::vector<int> W, screen_v, trial_v, tile_v, caps;
    std::vector<const void*> phi;
    std::vector<void*> e, ld;
    std::vector<int*> st;
    int mode = 0, precision = 0;
    bool tuned = false;  // recorded after the autotuner chose tile shapes and SM budgets
    // device allocations and frees seen when the graph was recorded: any later
    // one may have moved a buffer the graph holds, and the graph is re-recorded
    unsigned long long alloc_gen = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
    cudaGraphExec_t exec = nullptr;
    void release() {
        if (exec) cudaGraphExecDestroy(exec);
        for (cudaEvent_t ev : {fork, t0, t1})
            if (ev) cudaEventDestroy(ev);
        if (stream) cudaStreamDestroy(stream);
        exec = nullptr;
        stream = nullptr;
        fork = t0 = t1 = nullptr;
    }
};

std::mutex g_multi_mu;
std::vector<MultiPlan*> g_plans;

// drop every plan that uses context c (the caller holds g_multi_mu)
void drop_plans_locked(loaf_ctx* c) {
    for (auto it = g_plans.begin(); it != g_plans.end();) {
        if (std::find((*it)->ctxs.begin(), (*it)->ctxs.end(), c) != (*it)->ctxs.end()) {
            (*it)->release();
            delete *it;
            it = g_plans.erase(it);
        } else {
            ++it;
        }
    }
}

// drop every plan that uses context c (it is being destroyed, or its tile
// shapes changed)
void forget_plans(loaf_ctx* c) {
    std::lock_guard<std::mutex> lk(g_multi_mu);
    drop_plans_locked(c);
}

// The n branches of one multi-system graph: each context's batch on its own
// branch stream (the context's stream is swapped for the capture), outputs
// copied to the caller's buffers and the status flags to pinned host memory.
cudaGraphExec_t capture_multi(MultiPlan& P, const std::vector<int>& caps) {
    const int n = (int)P.ctxs.size();
    std::vector<cudaStream_t> saved(n);
    for (int k = 0; k < n; ++k) saved[k] = P.ctxs[k]->stream;
    auto restore = [&] {
        for (int k = 0; k < n; ++k) {
            P.ctxs[k]->stream = saved[k];
            P.ctxs[k]->grid_cap = 0;
        }
    };
    LOAF_CUDA(cudaStreamBeginCapture(P.stream, cudaStreamCaptureModeRelaxed));
    try {
        LOAF_CUDA(cudaEventRecord(P.fork, P.stream));
        for (int k = 0; k < n; ++k) {
            loaf_ctx* c = P.ctxs[k];
            c->stream = c->branch_stream;
            c->grid_cap = caps[k];
            LOAF_CUDA(cudaStreamWaitEvent(c->stream, P.fork, 0));
            const int W = P.W[k];
            double2* de = c->w_host_stage.as<double2>();
            double2* dld = de + W;
            int* dst = reinterpret_cast<int*>(dld + W);
            int* dflags = dst + W;
            LOAF_CUDA(cudaMemsetAsync(dflags, 0, 2 * sizeof(int), c->stream));
            energy_batch(c, W, static_cast<const double2*>(P.phi[k]), P.mode, P.precision, de, dld,
                         dst, dflags, dflags + 1);
            LOAF_CUDA(cudaMemcpyAsync(P.e[k], de, (size_t)W * sizeof(double2), cudaMemcpyDeviceToDevice,
                                      c->stream));
            if (P.ld[k])
                LOAF_CUDA(cudaMemcpyAsync(P.ld[k], dld, (size_t)W * sizeof(double2),
                                          cudaMemcpyDeviceToDevice, c->stream));
            if (P.st[k])
                LOAF_CUDA(cudaMemcpyAsync(P.st[k], dst, (size_t)W * sizeof(int), cudaMemcpyDeviceToDevice,
                                          c->stream));
            LOAF_CUDA(cudaMemcpyAsync(c->h_flags, dflags, 2 * sizeof(int), cudaMemcpyDeviceToHost,
                                      c->stream));
            LOAF_CUDA(cudaEventRecord(c->ev_join, c->stream));
            LOAF_CUDA(cudaStreamWaitEvent(P.stream, c->ev_join, 0));
            c->stream = saved[k];
            c->grid_cap = 0;
        }
    } catch (...) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(P.stream, &g);
        if (g) cudaGraphDestroy(g);
        restore();
        throw;
    }
    restore();
    cudaGraph_t graph = nullptr;
    LOAF_CUDA(cudaStreamEndCapture(P.stream, &graph));
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    LOAF_CUDA(ie);
    return exec;
}

float time_graph(MultiPlan& P, cudaGraphExec_t exec, int reps) {
    LOAF_CUDA(cudaGraphLaunch(exec, P.stream));
    LOAF_CUDA(cudaEventRecord(P.t0, P.stream));
    for (int r = 0; r < reps; ++r) LOAF_CUDA(cudaGraphLaunch(exec, P.stream));
    LOAF_CUDA(cudaEventRecord(P.t1, P.stream));
    LOAF_CUDA(cudaEventSynchronize(P.t1));
    float ms = 0.f;
    LOAF_CUDA(cudaEventElapsedTime(&ms, P.t0, P.t1));
    return ms / reps;
}

}  // namespace

extern "C" {

loaf_status walkers_energy_multi(loaf_ctx* const* ctxs, int n, const int* W, const void* const* phi,
                                 int mode, int precision, void* const* e_out, void* const* logdet_out,
                                 int* const* walker_status, int autotune, int* sm_caps) {
    if (!ctxs || n < 1 || !W || !phi || !e_out) return LOAF_ERR_ARG;
    loaf_ctx* c0 = ctxs[0];
    if (!c0) return LOAF_ERR_ARG;
    int flags[2] = {0, 0};
    loaf_status st = guarded(c0, [&] {
        LOAF_REQUIRE(mode == LOAF_MODE_LO, LOAF_ERR_UNSUPPORTED, "the multi-system launch runs the LO mode");
        for (int i = 0; i < n; ++i)
            if (ctxs[i]) drain_submitted(ctxs[i]);
        LOAF_REQUIRE(precision == LOAF_PREC_FP16X3 || precision == LOAF_PREC_BF16X3 ||
                         precision == LOAF_PREC_FP16X3_F64INV,
                     LOAF_ERR_UNSUPPORTED,
                     "the multi-system launch runs the split-precision path");
        for (int k = 0; k < n; ++k) {
            loaf_ctx* c = ctxs[k];
            LOAF_REQUIRE(c != nullptr && c->device == c0->device, LOAF_ERR_ARG,
                         "contexts must be non-NULL and on one device");
            for (int q = 0; q < k; ++q) LOAF_REQUIRE(ctxs[q] != c, LOAF_ERR_ARG, "a context appears twice");
            LOAF_REQUIRE(c->compressed, LOAF_ERR_NOT_READY, "lo_localize_compress has not been called");
            LOAF_REQUIRE(W[k] >= 1 && phi[k] && e_out[k], LOAF_ERR_ARG, "empty batch or NULL buffer");
            LOAF_REQUIRE(is_device_ptr(phi[k]) && is_device_ptr(e_out[k]) &&
                             (!logdet_out || !logdet_out[k] || is_device_ptr(logdet_out[k])) &&
                             (!walker_status || !walker_status[k] || is_device_ptr(walker_status[k])),
                         LOAF_ERR_ARG, "the multi-system launch takes device buffers only");
        }
        LOAF_CUDA(cudaSetDevice(c0->device));
        std::lock_guard<std::mutex> lk(g_multi_mu);
        // the plan of this signature (contexts, sizes, buffers, loaded trial,
        // screen and tile shapes), if one was recorded
        auto find_plan = [&]() -> MultiPlan* {
            for (MultiPlan* q : g_plans) {
                if ((int)q->ctxs.size() != n || q->mode != mode || q->precision != precision) continue;
                if (autotune && !q->tuned) continue;  // a tuned plan is recorded instead
                bool same = true;
                for (int k = 0; k < n && same; ++k)
                    same = q->ctxs[k] == ctxs[k] && q->W[k] == W[k] && q->phi[k] == phi[k] &&
                           q->e[k] == e_out[k] && q->ld[k] == (logdet_out ? logdet_out[k] : nullptr) &&
                           q->st[k] == (walker_status ? walker_status[k] : nullptr) &&
                           q->screen_v[k] == ctxs[k]->screen_version &&
                           q->trial_v[k] == ctxs[k]->trial_version && q->tile_v[k] == ctxs[k]->tile_version;
                if (same) return q;
            }
            return nullptr;
        };
        MultiPlan* P = find_plan();
        // one eager batch of system k on its context's stream (operands and
        // workspace are set up on the way; stage timers off)
        auto run_system = [&](int k) {
            loaf_ctx* c = ctxs[k];
            check_ready(c, W[k], phi[k], mode, precision);
            ensure_workspace(c, W[k], mode);
            double2* de = c->w_host_stage.as<double2>();
            double2* dld = de + W[k];
            int* dst = reinterpret_cast<int*>(dld + W[k]);
            int* dflags = dst + W[k];
            const bool prof = c->prof_on;
            c->prof_on = false;
            LOAF_CUDA(cudaMemsetAsync(dflags, 0, 2 * sizeof(int), c->stream));
            energy_batch(c, W[k], static_cast<const double2*>(phi[k]), mode, precision, de, dld, dst,
                         dflags, dflags + 1);
            c->prof_on = prof;
        };
        // an eager pass on each context sets up its operands and workspace, so
        // that recording a graph allocates nothing and waits on nothing
        auto eager_pass = [&] {
            for (int k = 0; k < n; ++k) {
                loaf_ctx* c = ctxs[k];
                if (!c->branch_stream) {
                    LOAF_CUDA(cudaStreamCreateWithFlags(&c->branch_stream, cudaStreamNonBlocking));
                    LOAF_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
                    LOAF_CUDA(cudaHostAlloc(&c->h_flags, 2 * sizeof(int), cudaHostAllocDefault));
                }
                run_system(k);
                LOAF_CUDA(cudaStreamSynchronize(c->stream));
            }
        };
        // Tile shapes of each system, timed with the GPU to itself: first the
        // largest LO chunk (the MMA's N: 256, 192, 128) with the Coulomb split of
        // the rule, then, with the best chunk, half and twice the rule's split.
        // A shape's result differs from another's only in the order of sums.
        auto tune_tiles = [&](int k) {
            loaf_ctx* c = ctxs[k];
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            LOAF_CUDA(cudaEventCreate(&e0));
            LOAF_CUDA(cudaEventCreate(&e1));
            auto time_shape = [&](int cap, int split) {
                c->tile_lo_cap = cap;
                c->tile_coul_split = split;
                run_system(k);  // builds the operands of this shape (untimed)
                LOAF_CUDA(cudaEventRecord(e0, c->stream));
                for (int r = 0; r < 3; ++r) run_system(k);
                LOAF_CUDA(cudaEventRecord(e1, c->stream));
                LOAF_CUDA(cudaEventSynchronize(e1));
                float ms = 0.f;
                LOAF_CUDA(cudaEventElapsedTime(&ms, e0, e1));
                return ms;
            };
            int best_cap = 256, best_split = 0;
            float best = time_shape(256, 0);
            for (int cap : {192, 128}) {
                const float ms = time_shape(cap, 0);
                if (ms < best) { best = ms; best_cap = cap; }
            }
            const int rule = coulomb_split_rule(c, W[k], precision);
            for (int split : {rule / 2, std::min(2 * rule, 16)}) {
                if (split < 1 || split == rule) continue;
                const float ms = time_shape(best_cap, split);
                if (ms < best) { best = ms; best_split = split; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            c->tile_lo_cap = best_cap;
            c->tile_coul_split = best_split;
            c->tile_version += 1;
            drop_plans_locked(c);  // recorded with the previous shapes
            LOAF_CUDA(cudaStreamSynchronize(c->stream));
        };
        if (!P && autotune) {
            // first call of this signature with the autotuner: tile shapes per
            // system (a new signature, since the tile versions change)
            eager_pass();
            for (int k = 0; k < n; ++k) tune_tiles(k);
            P = find_plan();
        }
        if (P && P->alloc_gen != devbuf_generation().load()) {
            // a buffer of some context may have moved since the graph was
            // recorded (another call grew a workspace, a setup call rebuilt the
            // operands): record it again with the SM budgets already chosen
            eager_pass();
            std::vector<bool> prof(n);
            for (int k = 0; k < n; ++k) { prof[k] = ctxs[k]->prof_on; ctxs[k]->prof_on = false; }
            cudaGraphExec_t ex = capture_multi(*P, P->caps);
            for (int k = 0; k < n; ++k) ctxs[k]->prof_on = prof[k];
            cudaGraphExecDestroy(P->exec);
            P->exec = ex;
            P->alloc_gen = devbuf_generation().load();
        }
        if (!P) {
            // first call of this signature: eager pass, then the graph is recorded
            eager_pass();
            P = new MultiPlan;
            g_plans.push_back(P);
            P->ctxs.assign(ctxs, ctxs + n);
            P->W.assign(W, W + n);
            P->phi.assign(phi, phi + n);
            P->e.assign(e_out, e_out + n);
            for (int k = 0; k < n; ++k) {
                P->ld.push_back(logdet_out ? logdet_out[k] : nullptr);
                P->st.push_back(walker_status ? walker_status[k] : nullptr);
                P->screen_v.push_back(ctxs[k]->screen_version);
                P->trial_v.push_back(ctxs[k]->trial_version);
                P->tile_v.push_back(ctxs[k]->tile_version);
            }
            P->mode = mode;
            P->precision = precision;
            LOAF_CUDA(cudaStreamCreateWithFlags(&P->stream, cudaStreamNonBlocking));
            LOAF_CUDA(cudaEventCreateWithFlags(&P->fork, cudaEventDisableTiming));
            LOAF_CUDA(cudaEventCreate(&P->t0));
            LOAF_CUDA(cudaEventCreate(&P->t1));
            std::vector<bool> prof(n);
            for (int k = 0; k < n; ++k) { prof[k] = ctxs[k]->prof_on; ctxs[k]->prof_on = false; }
            // candidate SM budgets: every system may fill the GPU, or each gets a
            // share proportional to its LO work (W x rows x M), rounded to SM pairs
            std::vector<std::vector<int>> cands{std::vector<int>(n, 0)};
            if (autotune && n > 1) {
                std::vector<double> work(n);
                double tot = 0.0;
                for (int k = 0; k < n; ++k) {
                    const MixedOps& mx = ctxs[k]->mix[mix_slot(precision)];
                    work[k] = (double)W[k] * (double)std::max<long>(mx.R, 1) * ctxs[k]->M;
                    tot += work[k];
                }
                std::vector<int> prop(n);
                for (int k = 0; k < n; ++k) {
                    int cap = (int)std::lround(c0->sm_count * work[k] / tot);
                    cap = std::max(8, std::min(c0->sm_count, (cap + 1) / 2 * 2));
                    prop[k] = cap;
                }
                cands.push_back(prop);
            }
            float best = 0.f;
            for (size_t q = 0; q < cands.size(); ++q) {
                cudaGraphExec_t ex = capture_multi(*P, cands[q]);
                const float ms = cands.size() > 1 ? time_graph(*P, ex, 3) : 0.f;
                if (!P->exec || ms < best) {
                    if (P->exec) cudaGraphExecDestroy(P->exec);
                    P->exec = ex;
                    P->caps = cands[q];
                    best = ms;
                } else {
                    cudaGraphExecDestroy(ex);
                }
            }
            for (int k = 0; k < n; ++k) ctxs[k]->prof_on = prof[k];
            P->alloc_gen = devbuf_generation().load();
            P->tuned = autotune != 0;
        }
        LOAF_CUDA(cudaGraphLaunch(P->exec, P->stream));
        LOAF_CUDA(cudaStreamSynchronize(P->stream));
        for (int k = 0; k < n; ++k) {
            flags[0] = std::max(flags[0], ctxs[k]->h_flags[0]);
            flags[1] = std::max(flags[1], ctxs[k]->h_flags[1]);
            if (sm_caps) sm_caps[k] = P->caps[k];
        }
    });
    if (st == LOAF_OK && flags[1]) {
        c0->err = "a tensor-core kernel gave up waiting on a pipeline barrier";
        return LOAF_ERR_TIMEOUT;
    }
    if (st == LOAF_OK && flags[0]) {
        c0->err = "at least one walker overlap is singular or non-finite";
        return flags[0] == LOAF_WALKER_SINGULAR ? LOAF_ERR_SINGULAR : LOAF_ERR_NAN;
    }
    return st;
}

loaf_status walkers_force_bias(loaf_ctx* c, int W, const void* phi, int precision, void* lbar_out,
                               void* logdet_out, int* walker_status) {
    if (!c) return LOAF_ERR_ARG;
    int flags[2] = {0, 0};
    loaf_status st = guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        check_ready(c, W, phi, LOAF_MODE_FULL, precision);
        LOAF_REQUIRE(lbar_out != nullptr, LOAF_ERR_ARG, "lbar_out is NULL");
        ensure_workspace(c, W, LOAF_MODE_FULL);
        const double2* dphi = stage_walkers(c, W, phi);
        double2* de = c->w_host_stage.as<double2>();
        double2* dld = de + W;
        int* dst = reinterpret_cast<int*>(dld + W);
        int* dflags = dst + W;
        LOAF_CUDA(cudaMemsetAsync(dflags, 0, 2 * sizeof(int), c->stream));
        const size_t X = (size_t)c->X;
        if (precision == LOAF_PREC_FP64) {
            stage_theta(c, W, dphi);
            run_coulomb_fp64(c, W, c->w_theta.as<double2>(), c->w_out.as<double2>());
            // rows g < X of the [W][X + 1] trace table
            LOAF_CUDA(cudaMemcpy2DAsync(lbar_out, X * sizeof(double2), c->w_part2.ptr, (X + 1) * sizeof(double2),
                                        X * sizeof(double2), W, cudaMemcpyDefault, c->stream));
        } else {
            run_theta_tc(c, W, dphi, precision);
            c->w_z.ensure((size_t)W * X * sizeof(double2));
            run_force_bias_mixed(c, W, precision, c->w_out.as<double2>(), c->w_z.as<double2>());
            LOAF_CUDA(cudaMemcpyAsync(lbar_out, c->w_z.ptr, (size_t)W * X * sizeof(double2), cudaMemcpyDefault,
                                      c->stream));
            flag_or_kernel<<<1, 1, 0, c->stream>>>(c->w_flag.as<int>(), dflags + 1);
            LOAF_LAUNCH_CHECK();
        }
        finalize_kernel<<<ceil_div(W, 128), 128, 0, c->stream>>>(
            W, c->nspin, c->sp[0].mult, c->nspin > 1 ? c->sp[1].mult : 0.0, c->e0, c->w_logdet.as<double2>(),
            c->w_status.as<int>(), nullptr, nullptr, nullptr, de, dld, dst, dflags);
        LOAF_LAUNCH_CHECK();
        deliver(c, logdet_out, dld, (size_t)W * sizeof(double2));
        deliver(c, walker_status, dst, (size_t)W * sizeof(int));
        LOAF_CUDA(cudaMemcpyAsync(flags, dflags, 2 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
    });
    if (st == LOAF_OK && flags[1]) {
        c->err = "a tensor-core kernel gave up waiting on a pipeline barrier";
        return LOAF_ERR_TIMEOUT;
    }
    if (st == LOAF_OK && flags[0]) {
        c->err = "at least one walker overlap is singular or non-finite";
        return flags[0] == LOAF_WALKER_SINGULAR ? LOAF_ERR_SINGULAR : LOAF_ERR_NAN;
    }
    return st;
}

loaf_status walkers_propagator(loaf_ctx* c, int W, const void* x, int precision, void* v_out) {
    if (!c) return LOAF_ERR_ARG;
    return guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        LOAF_REQUIRE(c->loaded, LOAF_ERR_NOT_READY, "ao_load_cholesky has not been called");
        LOAF_REQUIRE(W >= 1, LOAF_ERR_ARG, "W must be >= 1");
        LOAF_REQUIRE(x != nullptr && v_out != nullptr, LOAF_ERR_ARG, "x or v_out is NULL");
        LOAF_REQUIRE(precision != LOAF_PREC_TF32, LOAF_ERR_UNSUPPORTED,
                     "the TF32 precision is provided for the LO energy only");
        LOAF_REQUIRE(precision == LOAF_PREC_FP64 || precision == LOAF_PREC_FP16X3 ||
                         precision == LOAF_PREC_BF16X3 || precision == LOAF_PREC_FP16X3_F64INV,
                     LOAF_ERR_ARG, "unknown precision");
        const size_t xb = (size_t)W * c->X * sizeof(double2);
        const size_t vb = (size_t)W * c->M * c->M * sizeof(double2);
        const double2* dx = static_cast<const double2*>(x);
        if (!is_device_ptr(x)) {
            c->w_phi.ensure(xb);
            LOAF_CUDA(cudaMemcpyAsync(c->w_phi.ptr, x, xb, cudaMemcpyHostToDevice, c->stream));
            dx = c->w_phi.as<double2>();
        }
        double2* dv = static_cast<double2*>(v_out);
        const bool v_host = !is_device_ptr(v_out);
        if (v_host) {
            c->w_theta.ensure(vb);
            dv = c->w_theta.as<double2>();
        }
        run_propagator(c, W, dx, precision, dv);
        if (v_host) LOAF_CUDA(cudaMemcpyAsync(v_out, dv, vb, cudaMemcpyDeviceToHost, c->stream));
        int timeout = 0;
        if (precision != LOAF_PREC_FP64)
            LOAF_CUDA(cudaMemcpyAsync(&timeout, c->w_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        prof_collect(c);
        LOAF_REQUIRE(!timeout, LOAF_ERR_TIMEOUT, "a tensor-core kernel gave up waiting on a pipeline barrier");
    });
}

loaf_status walkers_energy_cas(loaf_ctx* c, int W, int N, const void* phi, int n_det, const int* dets,
                               const double* coeffs, void* e_out, void* logov_out, int* walker_status) {
    if (!c) return LOAF_ERR_ARG;
    int bad = 0;
    loaf_status st = guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        LOAF_REQUIRE(c->loaded, LOAF_ERR_NOT_READY, "ao_load_cholesky has not been called");
        LOAF_REQUIRE(c->compressed, LOAF_ERR_NOT_READY, "lo_localize_compress has not been called");
        LOAF_REQUIRE(c->closed && c->nspin == 1, LOAF_ERR_NOT_READY, "the CAS orbitals must be loaded as a closed shell");
        LOAF_REQUIRE(W >= 1, LOAF_ERR_ARG, "W must be >= 1");
        LOAF_REQUIRE(phi && dets && coeffs && e_out, LOAF_ERR_ARG, "phi, dets, coeffs or e_out is NULL");
        cas_check_dets(N, c->sp[0].N, n_det, dets);
        const size_t bytes = (size_t)W * c->M * N * sizeof(double2);
        const double2* dphi;
        if (is_device_ptr(phi)) {
            dphi = static_cast<const double2*>(phi);
        } else {
            c->w_phi.ensure(bytes);
            LOAF_CUDA(cudaMemcpyAsync(c->w_phi.ptr, phi, bytes, cudaMemcpyHostToDevice, c->stream));
            dphi = c->w_phi.as<double2>();
        }
        c->w_out.ensure((size_t)2 * W * sizeof(double2) + (size_t)W * sizeof(int));
        double2* de = c->w_out.as<double2>();
        double2* dlo = de + W;
        int* dst = reinterpret_cast<int*>(dlo + W);
        run_energy_cas(c, W, N, dphi, n_det, dets, coeffs, de, dlo, dst);
        deliver(c, e_out, de, (size_t)W * sizeof(double2));
        deliver(c, logov_out, dlo, (size_t)W * sizeof(double2));
        std::vector<int> hst(W);
        LOAF_CUDA(cudaMemcpyAsync(hst.data(), dst, (size_t)W * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        if (walker_status) {
            if (is_device_ptr(walker_status))
                LOAF_CUDA(cudaMemcpy(walker_status, dst, (size_t)W * sizeof(int), cudaMemcpyDeviceToDevice));
            else
                std::copy(hst.begin(), hst.end(), walker_status);
        }
        for (int v : hst)
            if (v != LOAF_WALKER_OK && bad == 0) bad = v;
    });
    if (st == LOAF_OK && bad) {
        c->err = "at least one walker's reference overlap is singular or non-finite";
        return bad == LOAF_WALKER_SINGULAR ? LOAF_ERR_SINGULAR : LOAF_ERR_NAN;
    }
    return st;
}

loaf_status walkers_pair_exchange(loaf_ctx* c, int W, const void* phi, int precision,
                                  void* e_pairs_out) {
    if (!c) return LOAF_ERR_ARG;
    return guarded(c, [&] {
        LOAF_CUDA(cudaSetDevice(c->device));
        check_ready(c, W, phi, LOAF_MODE_LO, precision);
        LOAF_REQUIRE(e_pairs_out != nullptr, LOAF_ERR_ARG, "e_pairs_out is NULL");
        ensure_workspace(c, W, LOAF_MODE_LO);
        const double2* dphi = stage_walkers(c, W, phi);
        if (precision == LOAF_PREC_FP64) {
            stage_theta(c, W, dphi);
            run_energy_fp64_lo(c, W, c->w_theta.as<double2>(), nullptr, c->w_part.as<double2>());
        } else {
            run_theta_tc(c, W, dphi, precision, prepare_lo_operands(c, LOAF_MODE_LO, precision));
            run_energy_mixed(c, W, LOAF_MODE_LO, precision, nullptr, nullptr,
                             c->w_part.as<double2>());
        }
        deliver(c, e_pairs_out, c->w_part.ptr, (size_t)loaf_num_pairs(c) * W * sizeof(double2));
        int timeout = 0;
        if (precision != LOAF_PREC_FP64)
            LOAF_CUDA(cudaMemcpyAsync(&timeout, c->w_flag.ptr, sizeof(int), cudaMemcpyDeviceToHost,
                                      c->stream));
        LOAF_CUDA(cudaStreamSynchronize(c->stream));
        prof_collect(c);
        LOAF_REQUIRE(!timeout, LOAF_ERR_TIMEOUT,
                     "a tensor-core kernel gave up waiting on a pipeline barrier");
    });
}

}  // extern "C"
