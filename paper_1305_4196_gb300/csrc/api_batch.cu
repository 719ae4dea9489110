// api_batch.cu - C ABI of ensembles of independent systems (include/mdgb_batch.h).
//
// Systems of at most BATCH_MAX_ATOMS atoms are grouped into size buckets; each
// bucket is one launch of k_batch_run (one CTA per system, all steps of the call),
// with the bucket's CTA size and cell range (chosen by md_batch_autotune, else a
// default).  The launches of a step call are captured once into a CUDA graph and
// replayed.  Larger systems are ordinary md_system instances, each on its own
// stream, stepped from a small pool of host threads while the launches run.
#include "mdgb.h"
#include "mdgb_batch.h"
#include "mdgb_batch_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

using namespace mdgb;

namespace {

constexpr int NBUCKET = 5;  // [.., 512), [512, 1024), [1024, 2048), [2048, 4096), [4096, 8192]
const int BUCKET_HI[NBUCKET] = {512, 1024, 2048, 4096, BATCH_MAX_ATOMS + 1};

int bucket_of(int64_t n) {
    for (int k = 0; k < NBUCKET; ++k)
        if (n < BUCKET_HI[k]) return k;
    return -1;
}

}  // namespace

struct md_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // capture only records; the legacy stream cannot capture
    cudaStream_t bucket_streams[NBUCKET] = {};  // one branch of the captured graph per size bucket
    cudaEvent_t fork_ev = nullptr, join_ev[NBUCKET] = {};
    int nsys = 0;
    std::vector<int64_t> n, a0;
    std::vector<double> box;  // 3 per system
    double r_cut = 0, skin = 0, dt = 0;
    md_params params{};
    double eps = 1, sigma = 1, mass = 1;
    PairTable pt{};
    int64_t ntot = 0;
    BatchState st{};
    double *d_pe = nullptr, *d_ke = nullptr;
    float* pe_atom = nullptr;
    double* d_aos = nullptr;  // N_total x 3 staging for AoS input/output
    struct Bucket {
        int threads = 256, R = 1;
        std::vector<int> ids;
        BatchSys* d_sys = nullptr;
        int nmax = 0, cmax = 0;
    };
    Bucket bk[NBUCKET];
    std::vector<int> path;  // 0: one CTA, 1: md_system
    std::vector<md_system*> big;
    std::vector<int> big_ids;
    std::vector<cudaStream_t> big_streams;
    bool has_state = false, have_forces = false;
    // graph of the launches of one md_batch_step call
    cudaGraphExec_t gexec = nullptr;
    int g_steps = -1, g_flags = -1;
    std::vector<void*> allocs;
    char msg[512] = "";
};

namespace {

int bfail(md_batch* b, int code, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->msg, sizeof(b->msg), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define BCK(call)                                                                                  \
    do {                                                                                           \
        cudaError_t e_ = (call);                                                                   \
        if (e_ != cudaSuccess) return bfail(b, MD_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

template <typename T>
int balloc(md_batch* b, T** p, size_t count) {
    *p = nullptr;
    void* q = nullptr;
    BCK(cudaMalloc(&q, std::max<size_t>(count, 1) * sizeof(T)));
    b->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return MD_OK;
}

// Geometry of one one-CTA system with cells at least r_cut / R wide (at most 16 per side).
BatchSys make_sys(const md_batch* b, int k, int R) {
    BatchSys y{};
    y.a0 = b->a0[k];
    y.id = k;
    y.n = (int)b->n[k];
    y.R = R;
    y.ncell = 1;
    for (int d = 0; d < 3; ++d) {
        const double L = b->box[3 * k + d];
        int nc = (int)std::floor(L * R / (b->r_cut * (1.0 + 1e-12)));
        nc = std::max(1, std::min(nc, 16));
        y.nc[d] = nc;
        y.L[d] = L;
        y.w[d] = L / nc;
        y.inv_w[d] = nc / L;
        y.wf[d] = (float)y.w[d];
        y.ncell *= nc;
    }
    return y;
}

int upload_bucket(md_batch* b, int k) {
    md_batch::Bucket& B = b->bk[k];
    if (B.ids.empty()) return MD_OK;
    std::vector<BatchSys> h;
    B.nmax = 0;
    B.cmax = 0;
    for (int id : B.ids) {
        h.push_back(make_sys(b, id, B.R));
        B.nmax = std::max(B.nmax, h.back().n);
        B.cmax = std::max(B.cmax, h.back().ncell);
    }
    B.nmax = (B.nmax + 7) & ~7;
    if (!B.d_sys && balloc(b, &B.d_sys, B.ids.size())) return MD_ERR_CUDA;
    BCK(cudaMemcpy(B.d_sys, h.data(), sizeof(BatchSys) * h.size(), cudaMemcpyHostToDevice));
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    return MD_OK;
}

bool bucket_fits(const md_batch* b, int k, int threads, int R) {
    int nmax = 0, cmax = 0;
    for (int id : b->bk[k].ids) {
        const BatchSys y = make_sys(b, id, R);
        nmax = std::max(nmax, y.n);
        cmax = std::max(cmax, y.ncell);
    }
    if (cmax > BATCH_MAX_CELLS) return false;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return threads <= BATCH_MAX_THREADS && batch_smem_bytes((nmax + 7) & ~7, cmax) + 8192 <= (size_t)optin;
}

// the launches of one step call: every non-empty bucket
void enqueue_buckets(md_batch* b, int n_steps, int flags, cudaStream_t s) {
    for (auto& B : b->bk) {
        if (B.ids.empty()) continue;
        launch_batch_run(B.d_sys, (int)B.ids.size(), b->st, b->pt, n_steps, flags, b->dt, B.threads, B.nmax, B.cmax,
                         b->d_pe, b->d_ke, b->pe_atom, s);
    }
}

int run_buckets(md_batch* b, int n_steps, int flags) {
    bool any = false;
    for (auto& B : b->bk) any |= !B.ids.empty();
    if (!any) return MD_OK;
    if (!(b->gexec && b->g_steps == n_steps && b->g_flags == flags)) {
        if (b->gexec) cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
        cudaGraph_t g = nullptr;
        // the buckets touch disjoint systems: one parallel branch each, so that they share the
        // GPU instead of running one after another
        BCK(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal));
        BCK(cudaEventRecord(b->fork_ev, b->cap_stream));
        for (int k = 0; k < NBUCKET; ++k) {
            md_batch::Bucket& B = b->bk[k];
            if (B.ids.empty()) continue;
            BCK(cudaStreamWaitEvent(b->bucket_streams[k], b->fork_ev, 0));
            launch_batch_run(B.d_sys, (int)B.ids.size(), b->st, b->pt, n_steps, flags, b->dt, B.threads, B.nmax,
                             B.cmax, b->d_pe, b->d_ke, b->pe_atom, b->bucket_streams[k]);
            BCK(cudaEventRecord(b->join_ev[k], b->bucket_streams[k]));
            BCK(cudaStreamWaitEvent(b->cap_stream, b->join_ev[k], 0));
        }
        BCK(cudaStreamEndCapture(b->cap_stream, &g));
        cudaError_t e = cudaGraphInstantiate(&b->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return bfail(b, MD_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
        b->g_steps = n_steps;
        b->g_flags = flags;
    }
    BCK(cudaGraphLaunch(b->gexec, b->stream));
    return MD_OK;
}

__global__ void k_aos_in(int64_t ntot, const double* __restrict__ pos, const double* __restrict__ vel,
                         const int32_t* __restrict__ sp, BatchState st) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= ntot) return;
    st.x[i] = pos[3 * i];
    st.y[i] = pos[3 * i + 1];
    st.z[i] = pos[3 * i + 2];
    st.vx[i] = vel[3 * i];
    st.vy[i] = vel[3 * i + 1];
    st.vz[i] = vel[3 * i + 2];
    st.ix[i] = st.iy[i] = st.iz[i] = 0;
    st.species[i] = sp ? sp[i] : 0;
}

__global__ void k_aos_out(int64_t lo, int64_t hi, BatchState st, int what, double* __restrict__ out,
                          int32_t* __restrict__ img) {
    const int64_t i = lo + blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= hi) return;
    if (what == 0) {
        out[3 * i] = st.x[i];
        out[3 * i + 1] = st.y[i];
        out[3 * i + 2] = st.z[i];
    } else if (what == 1) {
        out[3 * i] = st.vx[i];
        out[3 * i + 1] = st.vy[i];
        out[3 * i + 2] = st.vz[i];
    } else if (what == 2) {
        const double q = 2.3283064365386963e-10;  // 2^-32
        out[3 * i] = (double)st.fq[i] * q;
        out[3 * i + 1] = (double)st.fq[st.ntot + i] * q;
        out[3 * i + 2] = (double)st.fq[2 * st.ntot + i] * q;
    } else {
        img[3 * i] = st.ix[i];
        img[3 * i + 1] = st.iy[i];
        img[3 * i + 2] = st.iz[i];
    }
}

int check_batch_err(md_batch* b) {
    uint32_t e = 0;
    BCK(cudaMemcpy(&e, b->st.err, sizeof(uint32_t), cudaMemcpyDeviceToHost));
    if (!e) return MD_OK;
    if (e & ERR_NONFINITE) return bfail(b, MD_ERR_NONFINITE, "non-finite force or coordinate");
    if (e & ERR_ESCAPE) return bfail(b, MD_ERR_NONFINITE, "an atom moved more than one box length in a step");
    return bfail(b, MD_ERR_CUDA, "device error 0x%x", e);
}

// call f(k) for every large system from a pool of host threads; first nonzero code wins
template <typename F>
int for_big(md_batch* b, F&& f) {
    const int m = (int)b->big.size();
    if (m == 0) return MD_OK;
    // one host thread per core: each waits on its system's steps in turn
    const int nt = std::min(m, std::max(8, (int)std::thread::hardware_concurrency()));
    std::vector<int> rc(nt, MD_OK);
    std::vector<std::thread> th;
    for (int t = 0; t < nt; ++t)
        th.emplace_back([&, t]() {
            cudaSetDevice(b->device);
            for (int k = t; k < m; k += nt)
                if (rc[t] == MD_OK) rc[t] = f(k);
        });
    for (auto& x : th) x.join();
    for (int k = 0; k < m; ++k) {
        const int t = k % nt;
        if (rc[t] != MD_OK) {
            char buf[256] = "";
            md_last_error(b->big[k], buf, sizeof(buf));
            if (buf[0]) return bfail(b, rc[t], "system %d: %s", b->big_ids[k], buf);
        }
    }
    for (int t = 0; t < nt; ++t)
        if (rc[t] != MD_OK) return bfail(b, rc[t], "a system on the md_system path failed");
    return MD_OK;
}

}  // namespace

extern "C" {

int md_batch_create(int32_t n_systems, const int64_t* n_atoms, const double* boxes, double r_cut, double skin,
                    const md_params* p, md_batch** out) {
    if (!out) return MD_ERR_ARG;
    *out = nullptr;
    if (n_systems < 1 || !n_atoms || !boxes || !p || !(r_cut > 0.0) || !(skin >= 0.0)) return MD_ERR_ARG;
    if (p->n_species != 1 || p->precision != MD_MIXED || !p->eps || !p->sigma || !p->mass || !(p->dt > 0.0))
        return MD_ERR_ARG;
    md_batch* b = new md_batch();
    auto bail = [&](int code) {
        md_batch_destroy(b);
        return code;
    };
    cudaGetDevice(&b->device);
    b->stream = static_cast<cudaStream_t>(p->stream);
    if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) return bail(MD_ERR_CUDA);
    if (cudaEventCreateWithFlags(&b->fork_ev, cudaEventDisableTiming) != cudaSuccess) return bail(MD_ERR_CUDA);
    for (int k = 0; k < NBUCKET; ++k)
        if (cudaStreamCreateWithFlags(&b->bucket_streams[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join_ev[k], cudaEventDisableTiming) != cudaSuccess)
            return bail(MD_ERR_CUDA);
    b->nsys = n_systems;
    b->r_cut = r_cut;
    b->skin = skin;
    b->dt = p->dt;
    b->params = *p;
    b->eps = p->eps[0];
    b->sigma = p->sigma[0];
    b->mass = p->mass[0];
    b->params.eps = &b->eps;
    b->params.sigma = &b->sigma;
    b->params.mass = &b->mass;
    b->params.rcut = nullptr;
    b->params.list_kind = MD_LIST_FULL;
    // pair constants as the main path builds them (one species)
    b->pt.nsp = 1;
    b->pt.sig2_f[0] = (float)(b->sigma * b->sigma);
    b->pt.c48_f[0] = (float)(48.0 * b->eps * 2048.0);
    b->pt.c24_f[0] = (float)(24.0 * b->eps * 2048.0);
    b->pt.c4_f[0] = (float)(4.0 * b->eps);
    b->pt.rc2_f[0] = (float)(r_cut * r_cut);
    b->pt.rc2_d[0] = r_cut * r_cut;
    b->pt.mass[0] = b->mass;
    b->pt.hdtm[0] = (0.5 * p->dt) / b->mass;
    b->pt.hdtm_q[0] = b->pt.hdtm[0] * 0x1p-32;
    init_batch_kernels();
    b->n.assign(n_atoms, n_atoms + n_systems);
    b->box.assign(boxes, boxes + 3 * n_systems);
    b->a0.resize(n_systems);
    b->path.assign(n_systems, 0);
    for (int k = 0; k < n_systems; ++k) {
        if (b->n[k] < 0) return bail(MD_ERR_ARG);
        b->a0[k] = b->ntot;
        b->ntot += b->n[k];
        for (int d = 0; d < 3; ++d)
            if (!(boxes[3 * k + d] >= 2.0 * r_cut) || !std::isfinite(boxes[3 * k + d])) {
                bfail(b, MD_ERR_BOX_TOO_SMALL, "system %d: box side %g < 2 r_cut", k, boxes[3 * k + d]);
                return bail(MD_ERR_BOX_TOO_SMALL);
            }
        const int bu = bucket_of(b->n[k]);
        if (bu >= 0) {
            b->bk[bu].ids.push_back(k);
        } else {
            b->path[k] = 1;
            b->big_ids.push_back(k);
        }
    }
    // largest systems first within a bucket: CTAs start in index order, so the longest ones
    // are not left for the end of the launch
    for (auto& B : b->bk)
        std::stable_sort(B.ids.begin(), B.ids.end(), [&](int x, int y) { return b->n[x] > b->n[y]; });
    // FP64 decision band: the widest any system needs, for either cell divisor
    double band = 0.0;
    for (int k = 0; k < n_systems; ++k)
        for (int R = 1; R <= 2; ++R) {
            const BatchSys y = make_sys(b, k, R);
            band = std::max(band, cell_frame_cut_band(std::max(y.w[0], std::max(y.w[1], y.w[2])), R, r_cut));
        }
    b->pt.cut_band = (float)band;
    set_band_thresholds(b->pt);
    int rc;
    BatchState& st = b->st;
    st.ntot = b->ntot;
    if ((rc = balloc(b, &st.x, b->ntot)) || (rc = balloc(b, &st.y, b->ntot)) || (rc = balloc(b, &st.z, b->ntot)) ||
        (rc = balloc(b, &st.vx, b->ntot)) || (rc = balloc(b, &st.vy, b->ntot)) ||
        (rc = balloc(b, &st.vz, b->ntot)) || (rc = balloc(b, &st.ix, b->ntot)) ||
        (rc = balloc(b, &st.iy, b->ntot)) || (rc = balloc(b, &st.iz, b->ntot)) ||
        (rc = balloc(b, &st.species, b->ntot)) || (rc = balloc(b, &st.fq, 3 * (size_t)b->ntot)) ||
        (rc = balloc(b, &st.err, 1)) || (rc = balloc(b, &b->d_pe, n_systems)) ||
        (rc = balloc(b, &b->d_ke, n_systems)) || (rc = balloc(b, &b->pe_atom, b->ntot)) ||
        (rc = balloc(b, &b->d_aos, 3 * (size_t)b->ntot)))
        return bail(rc);
    if (cudaMemset(st.err, 0, sizeof(uint32_t)) != cudaSuccess) return bail(MD_ERR_CUDA);
    // default launch shapes; md_batch_autotune may change them
    const int def_threads[NBUCKET] = {128, 128, 256, 256, 512};
    for (int k = 0; k < NBUCKET; ++k) {
        b->bk[k].threads = def_threads[k];
        b->bk[k].R = 1;
        if (!b->bk[k].ids.empty() && !bucket_fits(b, k, b->bk[k].threads, 1)) {
            bfail(b, MD_ERR_CELL_OVERFLOW, "bucket %d does not fit in shared memory", k);
            return bail(MD_ERR_CELL_OVERFLOW);
        }
        if ((rc = upload_bucket(b, k))) return bail(rc);
    }
    // larger systems: ordinary systems on their own streams
    for (int k : b->big_ids) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return bail(MD_ERR_CUDA);
        b->big_streams.push_back(s);
        md_params q = b->params;
        q.stream = s;
        md_system* m = nullptr;
        if ((rc = md_create(b->n[k], &b->box[3 * k], r_cut, skin, &q, &m))) {
            bfail(b, rc, "system %d (%lld atoms) on the md_system path could not be created", k, (long long)b->n[k]);
            return bail(rc);
        }
        b->big.push_back(m);
    }
    *out = b;
    return MD_OK;
}

int md_batch_set_state(md_batch* b, const double* pos, const double* vel, const int32_t* species, int device_ptrs) {
    if (!b || !pos || !vel) return MD_ERR_ARG;
    const size_t n3 = 3 * (size_t)b->ntot;
    const double *P = pos, *V = vel;
    const int32_t* S = species;
    double* tmp = nullptr;
    int32_t* tsp = nullptr;
    if (!device_ptrs) {
        BCK(cudaMalloc(&tmp, sizeof(double) * 2 * std::max<size_t>(n3, 1)));
        BCK(cudaMemcpy(tmp, pos, sizeof(double) * n3, cudaMemcpyHostToDevice));
        BCK(cudaMemcpy(tmp + n3, vel, sizeof(double) * n3, cudaMemcpyHostToDevice));
        P = tmp;
        V = tmp + n3;
        if (species) {
            BCK(cudaMalloc(&tsp, sizeof(int32_t) * std::max<int64_t>(b->ntot, 1)));
            BCK(cudaMemcpy(tsp, species, sizeof(int32_t) * b->ntot, cudaMemcpyHostToDevice));
            S = tsp;
        }
    }
    if (b->ntot > 0) k_aos_in<<<(unsigned)((b->ntot + 255) / 256), 256, 0, b->stream>>>(b->ntot, P, V, S, b->st);
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->stream));
    int rc = for_big(b, [&](int k) {
        const int64_t o = 3 * b->a0[b->big_ids[k]];
        return md_set_state(b->big[k], P + o, V + o, S ? S + b->a0[b->big_ids[k]] : nullptr, 1);
    });
    if (tmp) cudaFree(tmp);
    if (tsp) cudaFree(tsp);
    if (rc) return rc;
    b->has_state = true;
    b->have_forces = false;
    return MD_OK;
}

int md_batch_step(md_batch* b, int32_t n_steps) {
    if (!b || n_steps < 0) return MD_ERR_ARG;
    if (!b->has_state) return bfail(b, MD_ERR_STATE, "no state: call md_batch_set_state first");
    if (n_steps == 0) return MD_OK;
    int rc = run_buckets(b, n_steps, b->have_forces ? BATCH_HAVE_FORCES : 0);
    if (rc) return rc;
    rc = for_big(b, [&](int k) { return md_step(b->big[k], n_steps); });
    BCK(cudaStreamSynchronize(b->stream));
    if (rc) return rc;
    if ((rc = check_batch_err(b))) return rc;
    b->have_forces = true;
    return MD_OK;
}

int md_batch_forces(md_batch* b, double* f_out, int device_ptrs) {
    if (!b) return MD_ERR_ARG;
    if (!b->has_state) return bfail(b, MD_ERR_STATE, "no state");
    int rc;
    if (!b->have_forces) {
        enqueue_buckets(b, 0, 0, b->stream);
        BCK(cudaGetLastError());
        b->have_forces = true;
    }
    if (!f_out) return MD_OK;
    double* dst = device_ptrs ? f_out : b->d_aos;
    for (int k = 0; k < b->nsys; ++k) {
        if (b->path[k] != 0 || b->n[k] == 0) continue;
        const int64_t lo = b->a0[k], hi = lo + b->n[k];
        k_aos_out<<<(unsigned)((hi - lo + 255) / 256), 256, 0, b->stream>>>(lo, hi, b->st, 2, dst, nullptr);
    }
    BCK(cudaGetLastError());
    BCK(cudaStreamSynchronize(b->stream));
    if ((rc = check_batch_err(b))) return rc;
    if (!device_ptrs) BCK(cudaMemcpy(f_out, b->d_aos, sizeof(double) * 3 * b->ntot, cudaMemcpyDeviceToHost));
    return for_big(b, [&](int k) {
        return md_forces(b->big[k], f_out + 3 * b->a0[b->big_ids[k]], device_ptrs);
    });
}

int md_batch_energies(md_batch* b, double* pe, double* ke) {
    if (!b || !pe || !ke) return MD_ERR_ARG;
    if (!b->has_state) return bfail(b, MD_ERR_STATE, "no state");
    int rc;
    enqueue_buckets(b, 0, BATCH_ENERGY, b->stream);
    BCK(cudaGetLastError());
    b->have_forces = true;
    std::vector<double> hp(b->nsys, 0.0), hk(b->nsys, 0.0);
    BCK(cudaMemcpyAsync(hp.data(), b->d_pe, sizeof(double) * b->nsys, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaMemcpyAsync(hk.data(), b->d_ke, sizeof(double) * b->nsys, cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if ((rc = check_batch_err(b))) return rc;
    rc = for_big(b, [&](int k) {
        double e = 0, q = 0;
        int r = md_energy_virial(b->big[k], &e, &q, nullptr);
        hp[b->big_ids[k]] = e;
        hk[b->big_ids[k]] = q;
        return r;
    });
    if (rc) return rc;
    std::copy(hp.begin(), hp.end(), pe);
    std::copy(hk.begin(), hk.end(), ke);
    return MD_OK;
}

int md_batch_get_state(md_batch* b, double* pos, double* vel, int32_t* image, int device_ptrs) {
    if (!b) return MD_ERR_ARG;
    if (!b->has_state) return bfail(b, MD_ERR_STATE, "no state");
    double* outs[2] = {pos, vel};
    for (int w = 0; w < 3; ++w) {
        double* o = w < 2 ? outs[w] : nullptr;
        if (w < 2 && !o) continue;
        if (w == 2 && !image) continue;
        double* dst = device_ptrs ? o : b->d_aos;
        int32_t* idst = device_ptrs ? image : reinterpret_cast<int32_t*>(b->d_aos);
        for (int k = 0; k < b->nsys; ++k) {
            if (b->path[k] != 0 || b->n[k] == 0) continue;
            const int64_t lo = b->a0[k], hi = lo + b->n[k];
            k_aos_out<<<(unsigned)((hi - lo + 255) / 256), 256, 0, b->stream>>>(lo, hi, b->st, w == 2 ? 3 : w, dst,
                                                                             idst);
        }
        BCK(cudaGetLastError());
        BCK(cudaStreamSynchronize(b->stream));
        if (!device_ptrs) {
            if (w < 2) BCK(cudaMemcpy(o, b->d_aos, sizeof(double) * 3 * b->ntot, cudaMemcpyDeviceToHost));
            else BCK(cudaMemcpy(image, b->d_aos, sizeof(int32_t) * 3 * b->ntot, cudaMemcpyDeviceToHost));
        }
    }
    return for_big(b, [&](int k) {
        const int64_t o = 3 * b->a0[b->big_ids[k]];
        return md_get_state(b->big[k], pos ? pos + o : nullptr, vel ? vel + o : nullptr, image ? image + o : nullptr,
                            device_ptrs);
    });
}

int md_batch_layout(md_batch* b, int32_t* path, int32_t* threads, int32_t* cell_range) {
    if (!b) return MD_ERR_ARG;
    for (int k = 0; k < b->nsys; ++k) {
        const int bu = b->path[k] == 0 ? bucket_of(b->n[k]) : -1;
        if (path) path[k] = b->path[k];
        if (threads) threads[k] = bu >= 0 ? b->bk[bu].threads : 0;
        if (cell_range) cell_range[k] = bu >= 0 ? b->bk[bu].R : 0;
    }
    return MD_OK;
}

int md_batch_autotune(md_batch* b, const char* cache_path) {
    if (!b) return MD_ERR_ARG;
    if (!b->has_state) return bfail(b, MD_ERR_STATE, "no state: the autotuner times real steps");
    cudaDeviceProp prop;
    BCK(cudaGetDeviceProperties(&prop, b->device));
    // cached choices for this GPU: bucket k -> (threads, R), or none for a bucket never tuned
    int cached[NBUCKET][2];
    for (int k = 0; k < NBUCKET; ++k) cached[k][0] = cached[k][1] = 0;
    if (cache_path) {
        FILE* f = std::fopen(cache_path, "r");
        if (f) {
            char buf[4096];
            const size_t len = std::fread(buf, 1, sizeof(buf) - 1, f);
            std::fclose(f);
            buf[len] = 0;
            const std::string s(buf);
            if (s.find(std::string("\"gpu\": \"") + prop.name + "\"") != std::string::npos) {
                for (int k = 0; k < NBUCKET; ++k) {
                    const std::string key = "\"bucket_" + std::to_string(k) + "\": [";
                    const size_t at = s.find(key);
                    int th = 0, R = 0;
                    if (at != std::string::npos && std::sscanf(s.c_str() + at + key.size(), "%d, %d", &th, &R) == 2 &&
                        (th == 128 || th == 256 || th == 512) && (R == 1 || R == 2)) {
                        cached[k][0] = th;
                        cached[k][1] = R;
                    }
                }
            }
        }
    }
    bool need = false, from_cache[NBUCKET] = {};
    for (int k = 0; k < NBUCKET; ++k) {
        md_batch::Bucket& B = b->bk[k];
        if (B.ids.empty()) continue;
        if (cached[k][0] && bucket_fits(b, k, cached[k][0], cached[k][1])) {
            B.threads = cached[k][0];
            B.R = cached[k][1];
            if (upload_bucket(b, k)) return MD_ERR_CUDA;
            from_cache[k] = true;
        } else {
            need = true;
        }
    }
    if (!need) return MD_OK;
    // time 10 steps per candidate on a copy of the state, restored afterwards
    const size_t n = (size_t)b->ntot;
    double* dsave = nullptr;
    int32_t* isave = nullptr;
    long long* fsave = nullptr;
    BCK(cudaMalloc(&dsave, sizeof(double) * 6 * std::max<size_t>(n, 1)));
    BCK(cudaMalloc(&isave, sizeof(int32_t) * 3 * std::max<size_t>(n, 1)));
    BCK(cudaMalloc(&fsave, sizeof(long long) * 3 * std::max<size_t>(n, 1)));
    double* D[6] = {b->st.x, b->st.y, b->st.z, b->st.vx, b->st.vy, b->st.vz};
    int32_t* I[3] = {b->st.ix, b->st.iy, b->st.iz};
    auto snap = [&](bool restore) {
        for (int c = 0; c < 6; ++c)
            cudaMemcpyAsync(restore ? D[c] : dsave + c * n, restore ? dsave + c * n : D[c], sizeof(double) * n,
                            cudaMemcpyDeviceToDevice, b->stream);
        for (int c = 0; c < 3; ++c)
            cudaMemcpyAsync(restore ? I[c] : isave + c * n, restore ? isave + c * n : I[c], sizeof(int32_t) * n,
                            cudaMemcpyDeviceToDevice, b->stream);
        cudaMemcpyAsync(restore ? b->st.fq : fsave, restore ? fsave : b->st.fq, sizeof(long long) * 3 * n,
                        cudaMemcpyDeviceToDevice, b->stream);
    };
    snap(false);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cand_t[3] = {128, 256, 512};
    std::string json = std::string("{\"gpu\": \"") + prop.name + "\"";
    for (int k = 0; k < NBUCKET; ++k) {
        md_batch::Bucket& B = b->bk[k];
        float best = 1e30f;
        int bt = B.threads, bR = B.R;
        if (!B.ids.empty() && !from_cache[k]) {
            for (int R = 1; R <= 2; ++R)
                for (int th : cand_t) {
                    if (!bucket_fits(b, k, th, R)) continue;
                    B.threads = th;
                    B.R = R;
                    if (upload_bucket(b, k)) return MD_ERR_CUDA;
                    launch_batch_run(B.d_sys, (int)B.ids.size(), b->st, b->pt, 1, 0, b->dt, B.threads, B.nmax, B.cmax,
                                     b->d_pe, b->d_ke, b->pe_atom, b->stream);  // warm-up
                    cudaEventRecord(e0, b->stream);
                    launch_batch_run(B.d_sys, (int)B.ids.size(), b->st, b->pt, 10, BATCH_HAVE_FORCES, b->dt,
                                     B.threads, B.nmax, B.cmax, b->d_pe, b->d_ke, b->pe_atom, b->stream);
                    cudaEventRecord(e1, b->stream);
                    BCK(cudaEventSynchronize(e1));
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, e0, e1);
                    snap(true);
                    if (ms < best) {
                        best = ms;
                        bt = th;
                        bR = R;
                    }
                }
            B.threads = bt;
            B.R = bR;
            if (upload_bucket(b, k)) return MD_ERR_CUDA;
            cached[k][0] = bt;
            cached[k][1] = bR;
        }
        if (cached[k][0])  // buckets never tuned are left out of the cache
            json += ", \"bucket_" + std::to_string(k) + "\": [" + std::to_string(cached[k][0]) + ", " +
                    std::to_string(cached[k][1]) + "]";
    }
    json += "}\n";
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    BCK(cudaStreamSynchronize(b->stream));
    cudaFree(dsave);
    cudaFree(isave);
    cudaFree(fsave);
    if (cudaMemset(b->st.err, 0, sizeof(uint32_t)) != cudaSuccess) return MD_ERR_CUDA;
    if (cache_path) {
        FILE* f = std::fopen(cache_path, "w");
        if (f) {
            std::fputs(json.c_str(), f);
            std::fclose(f);
        }
    }
    return MD_OK;
}

int md_batch_last_error(md_batch* b, char* buf, int64_t len) {
    if (!b || !buf || len <= 0) return MD_ERR_ARG;
    std::snprintf(buf, (size_t)len, "%s", b->msg);
    return MD_OK;
}

void md_batch_destroy(md_batch* b) {
    if (!b) return;
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    for (md_system* m : b->big) md_destroy(m);
    for (cudaStream_t s : b->big_streams) cudaStreamDestroy(s);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (int k = 0; k < NBUCKET; ++k) {
        if (b->bucket_streams[k]) cudaStreamDestroy(b->bucket_streams[k]);
        if (b->join_ev[k]) cudaEventDestroy(b->join_ev[k]);
    }
    if (b->fork_ev) cudaEventDestroy(b->fork_ev);
    for (void* p : b->allocs) cudaFree(p);
    delete b;
}

}  // extern "C"
