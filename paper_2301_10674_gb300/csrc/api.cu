// C ABI of the free-surface LBM / DEM step (declared in include/fslbm.h):
// parameter checks, device buffers, and the per-step kernel sequence.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "fslbm_dev.cuh"
#include "mlp_dev.cuh"

namespace fsl {
void mlp_from_bf16_host(const uint16_t* w, MlpBf16& h);
void mlp_mirror_w1_host(const uint16_t* w, __nv_bfloat16* out);
void mlp_frag_host(const MlpBf16& h, const __nv_bfloat16* w1m, MlpFrag& G);
}

namespace fsl {
void launch_export_owner(const Dev& s, int* out, cudaStream_t st);
void launch_bed_height(const Dev& s, double phi_b, double* phi, double* h, cudaStream_t st);
void launch_water_depth(const Dev& s, double* bed, double* eta, double* out, cudaStream_t st);
int launch_bed_spectrum(const double* h, int nt, int nx, double* psd, double* work, double* peak3, cudaStream_t st);
}

using namespace fsl;

struct fslbm {
    Dev d;
    fslbm_params p;
    cudaStream_t st;
    int64_t steps;
    int last_parity;   // layout of the stored post-collision PDFs (1 initially)
    int have_prev;
    bool spheres_added;
    std::vector<void*> allocs;
    // one device allocation holds the buffers fslbm_create makes (the arena);
    // planning: the first pass of the creation only adds up their sizes
    char* arena;
    size_t arena_size, arena_off;
    bool planning;
    double* stage;     // n doubles of staging for export/import
    double* red;       // 8 doubles for reductions
    int host_err;
    size_t elem;
    // measurement hooks
    bool timing;
    std::vector<cudaEvent_t> ev;   // start/end pairs of stream-collide sweeps
    size_t ev_used;
    int64_t launches;
    unsigned long long* counts4;
    double* bed;                   // nx * nz + nx doubles: phi_b(x, z), then h_b(x)
    double* eta;                   // nx * ny + 2 doubles: surface elevation, then depth and mean h_b
    // flow-rate control: target bulk velocity, gain, steps between updates (0: off)
    double ctrl_target, ctrl_gain;
    int64_t ctrl_interval;
    MlpBf16* mlp_dev;              // operand copies of the learned normal
    unsigned long long* mlp_stats;
    MlpFrag* mlp_frag_dev;         // in-step weights in fragment order, mirror images included
    // side stream of the DEM half of a step (overlapped with the free-surface
    // conversion), and the events that fork it from and join it to st
    cudaStream_t side;
    cudaEvent_t ev_fork, ev_join;
    // CUDA graphs of one step per parity (replayed once the step's launch
    // sequence and parameters are settled; captured again when a parameter
    // the kernels receive changes)
    cudaGraph_t graph[2];
    cudaGraphExec_t gexec[2];
    cudaGraphNode_t gev[2][2];   // the sweep's two event-record nodes per graph
    cudaEvent_t ev_cap[2];       // the events they record when no timing is on
    int graph_launches[2];
    bool graph_dirty;
    bool graphs_on;
};

namespace {

template <class T>
T* dalloc(fslbm* s, size_t count, bool& ok) {
    if (!ok) return nullptr;
    void* ptr = nullptr;
    size_t bytes = count * sizeof(T);
    if (bytes == 0) bytes = sizeof(T);
    const size_t padded = (bytes + 255) & ~(size_t)255;
    if (s->planning) {
        s->arena_size += padded;
        return reinterpret_cast<T*>(static_cast<uintptr_t>(256));   // replaced by the second pass
    }
    if (s->arena && s->arena_off + padded <= s->arena_size) {
        T* part = reinterpret_cast<T*>(s->arena + s->arena_off);
        s->arena_off += padded;
        return part;
    }
    if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        ok = false;
        cudaGetLastError();
        return nullptr;
    }
    s->allocs.push_back(ptr);
    return static_cast<T*>(ptr);
}

void* dalloc_bytes(fslbm* s, size_t bytes, bool& ok) { return dalloc<uint8_t>(s, bytes, ok); }

int map_device_error(int bits) {
    if (bits & ERR_NAN) return FSLBM_ENAN;
    if (bits & (ERR_CAPACITY | ERR_HISTORY | ERR_DISPLACEMENT)) return FSLBM_ECAPACITY;
    if (bits & ERR_INVARIANT) return FSLBM_EINVARIANT;
    if (bits & ERR_TIMEOUT) return FSLBM_ETIMEOUT;
    return FSLBM_OK;
}

// waits for the stream, folds CUDA and device errors into the sticky code
int sync_check(fslbm* s) {
    cudaError_t e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
        if (!s->host_err) s->host_err = FSLBM_EDEVICE;
        return s->host_err;
    }
    int bits = 0;
    if (cudaMemcpy(&bits, s->d.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) {
        if (!s->host_err) s->host_err = FSLBM_EDEVICE;
        return s->host_err;
    }
    if (!s->host_err) s->host_err = map_device_error(bits);
    return s->host_err;
}

int launch_check(fslbm* s) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess && !s->host_err) s->host_err = FSLBM_EDEVICE;
    return s->host_err;
}

cudaMemcpyKind kind_to(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost; }
cudaMemcpyKind kind_from(int on_device) { return on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice; }

}  // namespace

extern "C" {

void fslbm_default_params(fslbm_params* p) {
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->struct_size = sizeof(fslbm_params);
    p->nx = p->ny = p->nz = 1;
    p->bc_flags = FSLBM_PERIODIC_X;
    p->omega = 1.0 / 0.51;
    p->rho_gas = 1.0;
    p->liquid_height = 0.0;
    p->storage = FSLBM_STORE_FP32;
    p->normal_model = 0;
    p->reconstruct_normal = 1;
    p->eps_conv = 1e-2;
    p->eps_normal = 1e-2;
    p->rho_p = 2.55;
    p->restitution = 0.88;
    p->friction = 0.5;
    p->poisson = 0.22;
    p->collision_time = 24.0;
    p->dem_substeps = 10;
    p->link_mass_correction = 1;
    p->lubrication = 1;
}

const char* fslbm_strerror(int code) {
    switch (code) {
    case FSLBM_OK: return "ok";
    case FSLBM_EINVAL: return "invalid argument";
    case FSLBM_ENOMEM: return "device allocation failed";
    case FSLBM_ECAPACITY: return "device list capacity exceeded";
    case FSLBM_ENAN: return "non-finite value in the state";
    case FSLBM_EDEVICE: return "CUDA runtime error";
    case FSLBM_ESTATE: return "call not valid in the current state";
    case FSLBM_EINVARIANT: return "liquid cell next to a gas cell";
    case FSLBM_ETIMEOUT: return "a bounded device wait gave up";
    default: return "unknown error";
    }
}

int fslbm_create(const fslbm_params* p, void* cuda_stream, fslbm** out) {
    if (!p || !out) return FSLBM_EINVAL;
    *out = nullptr;
    if (p->struct_size != sizeof(fslbm_params)) return FSLBM_EINVAL;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return FSLBM_EINVAL;
    const long long n = (long long)p->nx * p->ny * p->nz;
    if (n >= (1LL << 31)) return FSLBM_EINVAL;
    if (!(p->omega > 0.0 && p->omega < 2.0)) return FSLBM_EINVAL;
    if (!std::isfinite(p->sigma) || p->sigma < 0.0) return FSLBM_EINVAL;
    if (p->normal_model < 0 || p->normal_model > 1 || p->init_profile != 0) return FSLBM_EINVAL;
    if (p->storage < 0 || p->storage > 2) return FSLBM_EINVAL;
    if (p->link_mass_correction < 0 || p->link_mass_correction > 1) return FSLBM_EINVAL;
    if (p->excess_even < 0 || p->excess_even > 1 || p->lubrication < 0 || p->lubrication > 1) return FSLBM_EINVAL;
    if (p->galilean_correction < 0 || p->galilean_correction > 1 || p->link_mode < 0 || p->link_mode > 2)
        return FSLBM_EINVAL;
    if (p->dem_substeps < 1 || !(p->restitution > 0.0 && p->restitution <= 1.0)) return FSLBM_EINVAL;
    if (!(p->collision_time > 0.0) || !(p->rho_p > 0.0) || !(p->rho_gas > 0.0)) return FSLBM_EINVAL;
    if (!(p->poisson >= 0.0 && p->poisson < 1.0) || !(p->friction >= 0.0)) return FSLBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(p->g[a])) return FSLBM_EINVAL;
    if (!std::isfinite(p->liquid_height) || p->eps_conv < 0.0 || p->eps_normal < 0.0) return FSLBM_EINVAL;

    fslbm* s = new (std::nothrow) fslbm();
    if (!s) return FSLBM_ENOMEM;
    s->p = *p;
    s->st = static_cast<cudaStream_t>(cuda_stream);
    s->steps = 0;
    s->last_parity = 1;
    s->have_prev = 0;
    s->spheres_added = false;
    s->host_err = 0;
    s->timing = false;
    s->ev_used = 0;
    s->launches = 0;
    s->counts4 = nullptr;
    s->bed = nullptr;
    s->eta = nullptr;
    s->ctrl_target = s->ctrl_gain = 0.0;
    s->ctrl_interval = 0;
    s->mlp_dev = nullptr;
    s->mlp_stats = nullptr;
    s->mlp_frag_dev = nullptr;
    s->d.mlp_frag = nullptr;
    s->d.mlp_mirror = 0;
    s->side = nullptr;
    s->ev_fork = s->ev_join = nullptr;
    for (int k = 0; k < 2; ++k) {
        s->graph[k] = nullptr;
        s->gexec[k] = nullptr;
        s->gev[k][0] = s->gev[k][1] = nullptr;
        s->ev_cap[k] = nullptr;
        s->graph_launches[k] = 0;
    }
    s->graph_dirty = false;
    // a stream can be captured unless it is the legacy default stream
    s->graphs_on = cuda_stream != nullptr && static_cast<cudaStream_t>(cuda_stream) != cudaStreamLegacy;
    Dev& d = s->d;
    std::memset(&d, 0, sizeof(d));
    d.nx = p->nx; d.ny = p->ny; d.nz = p->nz;
    d.per_x = (p->bc_flags & FSLBM_PERIODIC_X) ? 1 : 0;
    d.per_y = (p->bc_flags & FSLBM_PERIODIC_Y) ? 1 : 0;
    d.per_z = (p->bc_flags & FSLBM_PERIODIC_Z) ? 1 : 0;
    d.n = n;
    for (int q = 0; q < 27; ++q) {
        const long long off = fsl::cx(q) + (long long)p->nx * fsl::cy(q) + (long long)p->nx * p->ny * fsl::cz(q);
        d.pull_off[q] = (long long)fsl::opp(q) * n - off;
        d.push_off[q] = (long long)q * n + off;
    }
    d.omega = (float)p->omega;
    d.gx = (float)p->g[0]; d.gy = (float)p->g[1]; d.gz = (float)p->g[2];
    d.gxd = p->g[0]; d.gyd = p->g[1]; d.gzd = p->g[2];
    d.rho_gas = (float)p->rho_gas;
    d.sigma = (float)p->sigma;
    d.eps_conv = (float)p->eps_conv;
    d.eps_normal = (float)p->eps_normal;
    d.recon_normal = p->reconstruct_normal;
    d.excess_even = p->excess_even;
    d.galilean = p->galilean_correction;
    d.link_corr = p->link_mass_correction;
    d.idx32 = 27LL * n < (1LL << 32) ? 1 : 0;
    // fluid-side particle links need the pair kernels (nx even, 32-bit
    // indices, no Galilean correction) and the 32-cell type bit words
    d.links_fused = (p->link_mode == 2 && d.idx32 && p->nx % 32 == 0 && !p->galilean_correction) ? 1 : 0;
    d.nsegx = (p->nx + fsl::BED_SEG - 1) / fsl::BED_SEG;
    d.wait_limit = WAIT_LIMIT_DEFAULT;
    d.storage = p->storage;
    d.rho_p = p->rho_p;
    d.restitution = p->restitution;
    d.friction = p->friction;
    d.poisson = p->poisson;
    d.collision_time = p->collision_time;
    const double le = std::log(p->restitution);
    const double pi = 3.14159265358979323846;
    d.kn_coef = (pi * pi + le * le) / (p->collision_time * p->collision_time);
    d.dn_coef = -2.0 * le / p->collision_time;
    d.kt_ratio = 2.0 * (1.0 - p->poisson) / (2.0 - p->poisson);
    d.dem_substeps = p->dem_substeps;
    d.lub = p->lubrication;
    d.lub_mu = (1.0 / p->omega - 0.5) / 3.0;
    s->elem = p->storage == FSLBM_STORE_FP32 ? 4 : 2;

    // The buffers of the run are parts of one device allocation: the section
    // below runs twice, first adding up the sizes, then handing out 256-byte
    // aligned parts of the arena (one allocation and one release instead of
    // about eighty; buffers made later use cudaMalloc).
    int* counts = nullptr;
    double* dd = nullptr;
    float* href = nullptr;
    auto alloc_all = [&](bool& ok) {
        d.f = dalloc_bytes(s, (size_t)27 * n * s->elem, ok);
        d.fs = dalloc_bytes(s, (size_t)27 * n * s->elem, ok);
        d.flags = dalloc<uint8_t>(s, n + 4, ok);   // word-granular atomics on the last bytes
        d.mass = dalloc<float>(s, n, ok);
        d.phi = dalloc<float>(s, n, ok);
        d.ru = dalloc<float4>(s, n, ok);
        d.nrm = dalloc<float4>(s, n, ok);
        d.nrm1 = dalloc<float4>(s, n, ok);
        d.owner = dalloc<int>(s, n, ok);
        d.conv = dalloc<uint8_t>(s, n, ok);
        d.exscale = dalloc<float>(s, n, ok);
        long long cap = p->capacity_interface > 0 ? p->capacity_interface : n / 4 + 4096;
        if (cap > n) cap = n;
        d.wl_cap = (int)cap;
        d.nl_cap = (int)cap;
        d.wl = dalloc<int>(s, cap, ok);
        d.nl = dalloc<int>(s, cap, ok);
        d.cl = dalloc<int>(s, cap, ok);
        long long tcap = n / 8 + 4096;
        if (tcap > n) tcap = n;
        d.tl_cap = (int)tcap;
        d.tl = dalloc<int>(s, tcap, ok);
        d.sl_cap = (int)n;
        d.sl = dalloc<int>(s, n, ok);
        d.fbits = dalloc<unsigned>(s, n / 32 + 1, ok);
        d.ibits = dalloc<unsigned>(s, n / 32 + 1, ok);
        d.sbits = dalloc<unsigned>(s, n / 32 + 1, ok);
        d.tiles = dalloc<int>(s, n / fsl::SP_TILE + 1, ok);
        {
            const long long nseg = (long long)d.nsegx * p->ny * p->nz;
            d.segflag = dalloc<uint8_t>(s, nseg + 4, ok);
            d.bseg = dalloc<int>(s, nseg + 1, ok);
        }
        d.tl_info = dalloc<int>(s, 2 * tcap, ok);
        counts = dalloc<int>(s, 16, ok);
        if (ok) {
            d.wl_count = counts;
            d.nl_count = counts + 1;
            d.tl_count = counts + 2;
            d.zmax_cell = counts + 3;
            d.err = counts + 4;
            d.act_count = counts + 5;
            d.dl_count = counts + 6;
            d.sl_count = counts + 7;
            d.tile_count = counts + 8;
            d.bseg_count = counts + 9;
            d.cl_count = counts + 10;
            d.rtail_count = counts + 11;
        }
        dd = dalloc<double>(s, 4, ok);
        if (ok) {
            d.pool = dd;
            d.pool_share = dd + 1;
        }
        d.viol = dalloc<unsigned long long>(s, 1, ok);
        d.fixkey = dalloc<unsigned long long>(s, n, ok);
        d.fixowner = dalloc<int>(s, n, ok);
        long long pc = p->capacity_particles > 0 ? p->capacity_particles : 65536;
        d.np_cap = (int)pc;
        d.X = dalloc<double>(s, 3 * pc, ok); d.U = dalloc<double>(s, 3 * pc, ok); d.W = dalloc<double>(s, 3 * pc, ok);
        for (int k = 0; k < 2; ++k) {
            d.dem_dx[k] = dalloc<float>(s, 3 * pc, ok);
            d.dem_du[k] = dalloc<float>(s, 3 * pc, ok);
            d.dem_dw[k] = dalloc<float>(s, 3 * pc, ok);
        }
        d.nb_d0 = dalloc<float4>(s, pc * NB_SLOTS, ok);
        d.dem_wall = dalloc<float>(s, 6 * pc, ok);
        d.dem_c = dalloc<float4>(s, pc, ok);
        d.Faf = dalloc<float>(s, 3 * pc, ok);
        d.Taf = dalloc<float>(s, 3 * pc, ok);
        d.R = dalloc<double>(s, pc, ok); d.M = dalloc<double>(s, pc, ok); d.I = dalloc<double>(s, pc, ok);
        d.fixed = dalloc<uint8_t>(s, pc, ok);
        d.Xr = dalloc<float4>(s, pc, ok);
        d.Xi = dalloc<int4>(s, pc, ok);
        d.Xfr = dalloc<float4>(s, pc, ok);
        d.Uf = dalloc<float4>(s, pc, ok);
        d.Wf = dalloc<float4>(s, pc, ok);
        d.Fh = dalloc<double>(s, 3 * pc, ok); d.Th = dalloc<double>(s, 3 * pc, ok);
        d.Fp = dalloc<double>(s, 3 * pc, ok); d.Tp = dalloc<double>(s, 3 * pc, ok);
        d.Fa = dalloc<double>(s, 3 * pc, ok); d.Ta = dalloc<double>(s, 3 * pc, ok);
        d.hist_partner = dalloc<int>(s, pc * HIST_SLOTS, ok);
        d.nb = dalloc<int>(s, pc * NB_SLOTS, ok);
        d.nb_count = dalloc<int>(s, pc, ok);
        d.hist_xi = dalloc<float>(s, pc * HIST_SLOTS * 3, ok);
        d.g_of = dalloc<int>(s, pc, ok);
        d.Xm = dalloc<double>(s, 3 * pc, ok);
        d.margin = dalloc<float>(s, pc, ok);
        d.shared = dalloc<int>(s, pc, ok);
        d.act = dalloc<int>(s, pc, ok);
        d.dirty = dalloc<uint8_t>(s, n + 4, ok);
        d.scratch_a = dalloc<uint8_t>(s, n, ok);
        d.scratch_b = dalloc<uint8_t>(s, n, ok);
        const long long dcap = n;   // the first re-map may touch every cell of the bed
        d.dl_cap = (int)dcap;
        d.dl = dalloc<int>(s, dcap, ok);
        d.g_list = dalloc<int>(s, pc, ok);
        s->stage = dalloc<double>(s, n > 8 ? n : 8, ok);
        s->red = dalloc<double>(s, 8, ok);
        d.rpart = dalloc<double>(s, 8 * (size_t)reduce_blocks(d), ok);
        d.rtail = dalloc<double>(s, 8 * REDUCE_TAIL_BLOCKS, ok);
        href = p->storage != FSLBM_STORE_FP32 ? dalloc<float>(s, p->nz, ok) : nullptr;
    };
    s->arena = nullptr;
    s->arena_size = s->arena_off = 0;
    s->planning = true;
    bool ok = true;
    alloc_all(ok);
    s->planning = false;
    void* arena = nullptr;
    if (cudaMalloc(&arena, s->arena_size) == cudaSuccess) {
        s->arena = static_cast<char*>(arena);
        s->allocs.push_back(arena);
    } else {
        cudaGetLastError();   // the second pass allocates buffer by buffer
    }
    ok = true;
    alloc_all(ok);
    if (ok && (cudaStreamCreateWithFlags(&s->side, cudaStreamNonBlocking) != cudaSuccess ||
               cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
               cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess)) {
        cudaGetLastError();
        ok = false;
    }
    if (!ok) {
        fslbm_destroy(s);
        return FSLBM_ENOMEM;
    }
    cudaStream_t st = s->st;
    std::vector<float> href_h;
    if (href) {
        // reference of the 16-bit stored values: the hydrostatic density of
        // the flat initial surface, delta(z) = rho_gas exp(3 |g_z| (H - z_c)) - 1
        // (H clamped to the lattice), so that a stored value holds the
        // deviation from the liquid at rest and FP16/BF16 rounding acts on
        // the flow, not on the hydrostatic head
        const double H = std::min(std::max(p->liquid_height, 0.0), (double)p->nz);
        href_h.resize(p->nz);
        for (int z = 0; z < p->nz; ++z)
            href_h[z] = (float)(p->rho_gas * std::exp(3.0 * std::fabs(p->g[2]) * (H - (z + 0.5))) - 1.0);
        cudaMemcpyAsync(href, href_h.data(), sizeof(float) * p->nz, cudaMemcpyHostToDevice, st);
        d.href = href;
    }
    cudaMemsetAsync(d.f, 0, (size_t)27 * n * s->elem, st);
    cudaMemsetAsync(d.fs, 0, (size_t)27 * n * s->elem, st);
    cudaMemsetAsync(d.conv, 0, n, st);
    cudaMemsetAsync(d.exscale, 0, n * sizeof(float), st);
    cudaMemsetAsync(d.nrm1, 0, n * sizeof(float4), st);
    cudaMemsetAsync(counts, 0, 16 * sizeof(int), st);
    cudaMemsetAsync(dd, 0, 4 * sizeof(double), st);
    cudaMemsetAsync(d.viol, 0, sizeof(unsigned long long), st);
    cudaMemsetAsync(d.dirty, 0, n + 4, st);
    cudaMemsetAsync(d.fixowner, 0xff, n * sizeof(int), st);
    cudaMemsetAsync(d.segflag, 0, (size_t)d.nsegx * p->ny * p->nz + 4, st);
    launch_init_flat(d, p->liquid_height, st);
    launch_classify(d, st);
    launch_normals(d, d.nrm, st);
    if (launch_check(s) || sync_check(s)) {
        int e = s->host_err;
        fslbm_destroy(s);
        return e ? e : FSLBM_EDEVICE;
    }
    *out = s;
    return FSLBM_OK;
}

int fslbm_add_spheres(fslbm* s, int64_t n, const double* xyz, const double* radius, const uint8_t* fixed,
                      int on_device) {
    if (!s || n < 0 || (n > 0 && (!xyz || !radius))) return FSLBM_EINVAL;
    if (s->spheres_added || s->steps > 0) return FSLBM_ESTATE;
    if (n > s->d.np_cap) return FSLBM_ECAPACITY;
    Dev& d = s->d;
    std::vector<double> X(3 * n), R(n);
    std::vector<uint8_t> F(n, 0);
    if (n > 0) {
        cudaMemcpyKind k = on_device ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost;
        if (cudaMemcpy(X.data(), xyz, sizeof(double) * 3 * n, k) != cudaSuccess ||
            cudaMemcpy(R.data(), radius, sizeof(double) * n, k) != cudaSuccess ||
            (fixed && cudaMemcpy(F.data(), fixed, n, k) != cudaSuccess)) {
            cudaGetLastError();
            return FSLBM_EINVAL;
        }
    }
    const int L[3] = {d.nx, d.ny, d.nz};
    const int per[3] = {d.per_x, d.per_y, d.per_z};
    double rmax = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        if (!(R[i] > 0.0) || !std::isfinite(R[i])) return FSLBM_EINVAL;
        for (int a = 0; a < 3; ++a) {
            double v = X[3 * i + a];
            if (!std::isfinite(v)) return FSLBM_EINVAL;
            if (per[a]) {
                if (R[i] >= 0.5 * L[a]) return FSLBM_EINVAL;
                v -= L[a] * std::floor(v / L[a]);
                X[3 * i + a] = v;
            }
        }
        if (R[i] > rmax) rmax = R[i];
    }
    // particle grid: cells at least one diameter plus a skin wide
    const double h = 2.0 * rmax + 1.0;
    int gn[3];
    double gh[3];
    for (int a = 0; a < 3; ++a) {
        gn[a] = (int)std::floor(L[a] / h);
        if (gn[a] < 1) gn[a] = 1;
        gh[a] = (double)L[a] / gn[a];
    }
    d.gnx = gn[0]; d.gny = gn[1]; d.gnz = gn[2];
    d.ghx = gh[0]; d.ghy = gh[1]; d.ghz = gh[2];
    d.r_max = rmax;
    const long long G = (long long)gn[0] * gn[1] * gn[2];
    bool ok = true;
    d.g_count = dalloc<int>(s, G, ok);
    d.g_start = dalloc<int>(s, G, ok);
    d.g_cursor = dalloc<int>(s, G, ok);
    if (!ok) return FSLBM_ENOMEM;
    d.np = (int)n;
    cudaStream_t st = s->st;
    if (n > 0) {
        cudaMemcpyAsync(d.X, X.data(), sizeof(double) * 3 * n, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d.R, R.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(d.fixed, F.data(), n, cudaMemcpyHostToDevice, st);
        launch_particles_add(d, 0, (int)n, st);
        launch_classify(d, st);
        launch_normals(d, d.nrm, st);
    }
    s->spheres_added = true;
    s->graph_dirty = true;
    launch_check(s);
    return sync_check(s);
}

int fslbm_init_surface(fslbm* s, const double* height_xy, int on_device) {
    if (!s || !height_xy) return FSLBM_EINVAL;
    if (s->steps > 0) return FSLBM_ESTATE;
    Dev& d = s->d;
    const size_t cnt = (size_t)d.nx * d.ny;
    cudaMemcpyAsync(s->stage, height_xy, cnt * sizeof(double), kind_from(on_device), s->st);
    launch_init_surface(d, s->stage, s->st);
    launch_classify(d, s->st);
    launch_normals(d, d.nrm, s->st);
    launch_check(s);
    return sync_check(s);
}

// Enqueues the launches of one step of the given parity on s->st (and the
// DEM half on the side stream); returns the number of kernels. Under graph
// capture the sweep's two timing events are recorded as external
// event-record nodes of the placeholder events, retargeted at each replay.
static int enqueue_step(fslbm* s, int parity, bool capturing) {
    Dev& d = s->d;
    cudaStream_t st = s->st;
    if (d.np > 0) {
        cudaMemsetAsync(d.Fh, 0, sizeof(double) * 3 * d.np, st);
        cudaMemsetAsync(d.Th, 0, sizeof(double) * 3 * d.np, st);
    }
    int nl = 0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (capturing) {
        e0 = s->ev_cap[0];
        e1 = s->ev_cap[1];
        cudaEventRecordWithFlags(e0, st, cudaEventRecordExternal);
    } else if (s->timing) {
        if (s->ev_used + 2 > s->ev.size()) {
            for (int j = 0; j < 64; ++j) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                s->ev.push_back(e);
            }
        }
        e0 = s->ev[s->ev_used++];
        e1 = s->ev[s->ev_used++];
        cudaEventRecord(e0, st);
    }
    nl += launch_stream_collide(d, parity, st, d.np > 0 ? s->ev_fork : nullptr);
    if (capturing)
        cudaEventRecordWithFlags(e1, st, cudaEventRecordExternal);
    else if (s->timing)
        cudaEventRecord(e1, st);
    if (d.np > 0) {
        // the DEM half on the side stream, from the end of the link pass:
        // beside the liquid kernels and the conversion.
        // Those read no particle state, and the DEM no fluid state.
        cudaStreamWaitEvent(s->side, s->ev_fork, 0);
        nl += launch_dem(d, s->have_prev, s->side);
        cudaEventRecord(s->ev_join, s->side);
    }
    nl += launch_conversion(d, parity, st);
    if (d.np > 0) {
        cudaStreamWaitEvent(st, s->ev_join, 0);
        nl += launch_remap(d, parity, st);
    }
    nl += launch_classify(d, st);
    nl += launch_pool_spread(d, st);
    nl += launch_normals(d, d.nrm, st);
    return nl;
}

static void drop_graph(fslbm* s, int parity) {
    if (s->gexec[parity]) cudaGraphExecDestroy(s->gexec[parity]);
    if (s->graph[parity]) cudaGraphDestroy(s->graph[parity]);
    s->gexec[parity] = nullptr;
    s->graph[parity] = nullptr;
    s->gev[parity][0] = s->gev[parity][1] = nullptr;
}

// Captures the step of one parity into a graph; false if it cannot be (the
// stream is already being captured by the caller, or capture fails: graphs
// then stay off for this simulation).
static bool capture_step(fslbm* s, int parity) {
    drop_graph(s, parity);
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s->st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return false;
    }
    for (int k = 0; k < 2; ++k)
        if (!s->ev_cap[k] && cudaEventCreate(&s->ev_cap[k]) != cudaSuccess) {
            cudaGetLastError();
            s->graphs_on = false;
            return false;
        }
    if (cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        s->graphs_on = false;
        return false;
    }
    const int nl = enqueue_step(s, parity, true);
    cudaGraph_t g = nullptr;
    if (cudaStreamEndCapture(s->st, &g) != cudaSuccess || !g) {
        cudaGetLastError();
        if (g) cudaGraphDestroy(g);
        s->graphs_on = false;
        return false;
    }
    // the two event-record nodes, told apart by their placeholder event
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t k = 0; k < nn; ++k) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nodes[k], &t) != cudaSuccess || t != cudaGraphNodeTypeEventRecord) continue;
        cudaEvent_t e = nullptr;
        cudaGraphEventRecordNodeGetEvent(nodes[k], &e);
        if (e == s->ev_cap[0]) s->gev[parity][0] = nodes[k];
        if (e == s->ev_cap[1]) s->gev[parity][1] = nodes[k];
    }
    s->graph[parity] = g;
    if (!s->gev[parity][0] || !s->gev[parity][1] ||
        cudaGraphInstantiate(&s->gexec[parity], g, 0) != cudaSuccess) {
        cudaGetLastError();
        drop_graph(s, parity);
        s->graphs_on = false;
        return false;
    }
    s->graph_launches[parity] = nl;
    return true;
}

// Replays the graph of one parity; the sweep's events are retargeted at a
// fresh pair when timing is on.
static int replay_step(fslbm* s, int parity) {
    if (s->timing) {
        if (s->ev_used + 2 > s->ev.size()) {
            for (int j = 0; j < 64; ++j) {
                cudaEvent_t e;
                cudaEventCreate(&e);
                s->ev.push_back(e);
            }
        }
        cudaGraphExecEventRecordNodeSetEvent(s->gexec[parity], s->gev[parity][0], s->ev[s->ev_used++]);
        cudaGraphExecEventRecordNodeSetEvent(s->gexec[parity], s->gev[parity][1], s->ev[s->ev_used++]);
    } else {
        cudaGraphExecEventRecordNodeSetEvent(s->gexec[parity], s->gev[parity][0], s->ev_cap[0]);
        cudaGraphExecEventRecordNodeSetEvent(s->gexec[parity], s->gev[parity][1], s->ev_cap[1]);
    }
    cudaGraphLaunch(s->gexec[parity], s->st);
    return s->graph_launches[parity];
}

int fslbm_step(fslbm* s, int64_t n_steps) {
    if (!s || n_steps < 0) return FSLBM_EINVAL;
    if (s->host_err) return s->host_err;
    if (s->p.normal_model == 1 && !s->d.mlp) return FSLBM_ESTATE;
    Dev& d = s->d;
    cudaStream_t st = s->st;
    if (s->graph_dirty) {
        drop_graph(s, 0);
        drop_graph(s, 1);
        s->graph_dirty = false;
    }
    for (int64_t k = 0; k < n_steps; ++k) {
        const int parity = (int)(s->steps & 1);
        int nl = 0;
        // replay a graph of the step once its launch sequence is settled
        // (from the third step on: the first differs, and both parities have
        // then run once), unless the flow control changes the body force
        // between steps
        const bool graph = s->graphs_on && s->ctrl_interval == 0 && s->steps >= 2;
        if (graph && (s->gexec[parity] || capture_step(s, parity)))
            nl = replay_step(s, parity);
        else
            nl = enqueue_step(s, parity, false);
        s->last_parity = parity;
        s->have_prev = 1;
        s->steps++;
        if (s->ctrl_interval > 0 && s->steps % s->ctrl_interval == 0) {
            // flow-rate control: g_x += gain (U_target - U), U the fill-weighted
            // bulk velocity of the state just reached
            double r[8];
            launch_reduce(d, s->last_parity, s->red, st);
            nl += 2;
            cudaMemcpyAsync(r, s->red, sizeof(r), cudaMemcpyDeviceToHost, st);
            launch_check(s);
            if (sync_check(s)) return s->host_err;
            // kept within the range fslbm_set_body_force accepts
            double gx = d.gxd + s->ctrl_gain * (s->ctrl_target - r[4]);
            if (!std::isfinite(gx)) {
                s->host_err = FSLBM_ENAN;
                return s->host_err;
            }
            gx = gx > 1.0 ? 1.0 : (gx < -1.0 ? -1.0 : gx);
            d.gxd = gx;
            d.gx = (float)gx;
        }
        if (s->timing) s->launches += nl;
    }
    return launch_check(s);
}

int fslbm_get_fields(fslbm* s, uint32_t mask, void* const* dst, int dst_on_device) {
    if (!s || !dst) return FSLBM_EINVAL;
    Dev& d = s->d;
    cudaStream_t st = s->st;
    const long long n = d.n;
    int k = 0;
    for (int bit = 0; bit < 32; ++bit) {
        uint32_t b = 1u << bit;
        if (!(mask & b)) continue;
        void* out = dst[k++];
        if (!out) return FSLBM_EINVAL;
        switch (b) {
        case FSLBM_FIELD_PDF:
            for (int q = 0; q < 27; ++q) {
                // one direction at a time through the n-double staging buffer
                launch_export(d, s->last_parity, FSLBM_FIELD_PDF | (uint32_t)(q << 8), s->stage, st);
                cudaMemcpyAsync(static_cast<double*>(out) + (size_t)q * n, s->stage, n * sizeof(double),
                                kind_to(dst_on_device), st);
            }
            break;
        case FSLBM_FIELD_TYPE:
            launch_export_type(d, reinterpret_cast<uint8_t*>(s->stage), st);
            cudaMemcpyAsync(out, s->stage, n, kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_OWNER:
            launch_export_owner(d, reinterpret_cast<int*>(s->stage), st);
            cudaMemcpyAsync(out, s->stage, n * sizeof(int), kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_MASS:
        case FSLBM_FIELD_PHI:
        case FSLBM_FIELD_RHO:
            launch_export(d, s->last_parity, b, s->stage, st);
            cudaMemcpyAsync(out, s->stage, n * sizeof(double), kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_U:
        case FSLBM_FIELD_NORMAL:
            for (int a = 0; a < 3; ++a) {
                launch_export(d, s->last_parity, b | (uint32_t)(a << 8), s->stage, st);
                cudaMemcpyAsync(static_cast<double*>(out) + (size_t)a * n, s->stage, n * sizeof(double),
                                kind_to(dst_on_device), st);
            }
            break;
        case FSLBM_FIELD_P_X:
            cudaMemcpyAsync(out, d.X, sizeof(double) * 3 * d.np, kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_P_U:
            cudaMemcpyAsync(out, d.U, sizeof(double) * 3 * d.np, kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_P_OMEGA:
            cudaMemcpyAsync(out, d.W, sizeof(double) * 3 * d.np, kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_P_F:
            cudaMemcpyAsync(out, d.Fh, sizeof(double) * 3 * d.np, kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_P_T:
            cudaMemcpyAsync(out, d.Th, sizeof(double) * 3 * d.np, kind_to(dst_on_device), st);
            break;
        case FSLBM_FIELD_P_R:
            cudaMemcpyAsync(out, d.R, sizeof(double) * d.np, kind_to(dst_on_device), st);
            break;
        default:
            return FSLBM_EINVAL;
        }
    }
    launch_check(s);
    return sync_check(s);
}

int fslbm_set_fields(fslbm* s, uint32_t mask, const void* const* src, int src_on_device) {
    if (!s || !src) return FSLBM_EINVAL;
    Dev& d = s->d;
    cudaStream_t st = s->st;
    const long long n = d.n;
    int k = 0;
    for (int bit = 0; bit < 32; ++bit) {
        uint32_t b = 1u << bit;
        if (!(mask & b)) continue;
        const void* in = src[k++];
        if (!in) return FSLBM_EINVAL;
        switch (b) {
        case FSLBM_FIELD_PDF:
            for (int q = 0; q < 27; ++q) {
                cudaMemcpyAsync(s->stage, static_cast<const double*>(in) + (size_t)q * n, n * sizeof(double),
                                kind_from(src_on_device), st);
                launch_import_pdf(d, s->last_parity | (q << 8), s->stage, st);
            }
            launch_import_pdf(d, s->last_parity | (27 << 8), nullptr, st);
            break;
        case FSLBM_FIELD_MASS:
            cudaMemcpyAsync(s->stage, in, n * sizeof(double), kind_from(src_on_device), st);
            launch_import_mass(d, s->stage, st);
            launch_normals(d, d.nrm, st);
            break;
        case FSLBM_FIELD_P_U:
            cudaMemcpyAsync(d.U, in, sizeof(double) * 3 * d.np, kind_from(src_on_device), st);
            break;
        case FSLBM_FIELD_P_OMEGA:
            cudaMemcpyAsync(d.W, in, sizeof(double) * 3 * d.np, kind_from(src_on_device), st);
            break;
        default:
            return FSLBM_EINVAL;
        }
    }
    if (mask & (FSLBM_FIELD_P_U | FSLBM_FIELD_P_OMEGA)) launch_particle_copies(d, st);
    launch_check(s);
    return sync_check(s);
}

int fslbm_reduce(fslbm* s, double out[8]) {
    if (!s || !out) return FSLBM_EINVAL;
    launch_reduce(s->d, s->last_parity, s->red, s->st);
    cudaMemcpyAsync(out, s->red, 8 * sizeof(double), cudaMemcpyDeviceToHost, s->st);
    launch_check(s);
    return sync_check(s);
}

int fslbm_sync(fslbm* s) {
    if (!s) return FSLBM_EINVAL;
    launch_check(s);
    return sync_check(s);
}

int64_t fslbm_steps_done(const fslbm* s) { return s ? s->steps : -1; }
int64_t fslbm_num_spheres(const fslbm* s) { return s ? s->d.np : -1; }

int64_t fslbm_invariant_violations(fslbm* s) {
    if (!s) return -1;
    unsigned long long v = 0;
    launch_check_invariant(s->d, s->st);
    cudaStreamSynchronize(s->st);
    cudaMemcpy(&v, s->d.viol, sizeof(v), cudaMemcpyDeviceToHost);
    return (int64_t)v;
}

int fslbm_timing(fslbm* s, int on) {
    if (!s) return FSLBM_EINVAL;
    s->timing = on != 0;
    if (on) {
        cudaStreamSynchronize(s->st);
        s->ev_used = 0;
        s->launches = 0;
    }
    return launch_check(s);
}

int fslbm_timing_read(fslbm* s, double* sweep_ms, int64_t* sweeps, int64_t* kernel_launches) {
    if (!s) return FSLBM_EINVAL;
    int rc = sync_check(s);
    double total = 0.0;
    for (size_t k = 0; k + 1 < s->ev_used; k += 2) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, s->ev[k], s->ev[k + 1]) == cudaSuccess) total += ms;
    }
    if (sweep_ms) *sweep_ms = total;
    if (sweeps) *sweeps = (int64_t)(s->ev_used / 2);
    if (kernel_launches) *kernel_launches = s->launches;
    return rc;
}

int fslbm_cell_counts(fslbm* s, int64_t counts[4]) {
    if (!s || !counts) return FSLBM_EINVAL;
    if (!s->counts4) {
        bool ok = true;
        s->counts4 = dalloc<unsigned long long>(s, 4, ok);
        if (!ok) return FSLBM_ENOMEM;
    }
    launch_cell_counts(s->d, s->counts4, s->st);
    unsigned long long h[4] = {0, 0, 0, 0};
    cudaMemcpyAsync(h, s->counts4, sizeof(h), cudaMemcpyDeviceToHost, s->st);
    int rc = sync_check(s);
    for (int k = 0; k < 4; ++k) counts[k] = (int64_t)h[k];
    return rc;
}

int fslbm_set_body_force(fslbm* s, const double g[3]) {
    if (!s || !g) return FSLBM_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (!(g[a] == g[a]) || g[a] > 1.0 || g[a] < -1.0) return FSLBM_EINVAL;
    Dev& d = s->d;
    d.gxd = g[0]; d.gyd = g[1]; d.gzd = g[2];
    d.gx = (float)g[0]; d.gy = (float)g[1]; d.gz = (float)g[2];
    s->graph_dirty = true;
    return FSLBM_OK;
}

int fslbm_get_body_force(const fslbm* s, double g[3]) {
    if (!s || !g) return FSLBM_EINVAL;
    g[0] = s->d.gxd; g[1] = s->d.gyd; g[2] = s->d.gzd;
    return FSLBM_OK;
}

int fslbm_set_flow_control(fslbm* s, double target_u, double gain, int64_t interval) {
    if (!s || interval < 0 || !std::isfinite(target_u) || !std::isfinite(gain) || gain < 0.0) return FSLBM_EINVAL;
    s->ctrl_target = target_u;
    s->ctrl_gain = gain;
    s->ctrl_interval = interval;
    s->graph_dirty = true;
    return FSLBM_OK;
}

int fslbm_bed_height(fslbm* s, double phi_b, double* h, double* phi, int on_device) {
    if (!s || !h || !(phi_b > 0.0 && phi_b <= 1.0)) return FSLBM_EINVAL;
    if (s->host_err) return s->host_err;
    const Dev& d = s->d;
    const size_t nxz = (size_t)d.nx * d.nz;
    if (!s->bed) {
        bool ok = true;
        s->bed = dalloc<double>(s, nxz + d.nx, ok);
        if (!ok) return FSLBM_ENOMEM;
    }
    launch_bed_height(d, phi_b, s->bed, s->bed + nxz, s->st);
    const cudaMemcpyKind kind = kind_to(on_device);
    cudaMemcpyAsync(h, s->bed + nxz, d.nx * sizeof(double), kind, s->st);
    if (phi) cudaMemcpyAsync(phi, s->bed, nxz * sizeof(double), kind, s->st);
    launch_check(s);
    return sync_check(s);
}

int fslbm_transport_numbers(fslbm* s, double d50, double out[6]) {
    if (!s || !out || !(d50 > 0.0) || !std::isfinite(d50)) return FSLBM_EINVAL;
    if (s->host_err) return s->host_err;
    const Dev& d = s->d;
    const size_t nxz = (size_t)d.nx * d.nz, nxy = (size_t)d.nx * d.ny;
    bool ok = true;
    if (!s->bed) s->bed = dalloc<double>(s, nxz + d.nx, ok);
    if (!s->eta) s->eta = dalloc<double>(s, nxy + 2, ok);
    if (!ok) return FSLBM_ENOMEM;
    launch_water_depth(d, s->bed, s->eta, s->eta + nxy, s->st);
    launch_reduce(d, s->last_parity, s->red, s->st);
    double dep[2] = {0.0, 0.0}, red[8];
    cudaMemcpyAsync(dep, s->eta + nxy, sizeof(dep), cudaMemcpyDeviceToHost, s->st);
    cudaMemcpyAsync(red, s->red, sizeof(red), cudaMemcpyDeviceToHost, s->st);
    launch_check(s);
    const int rc = sync_check(s);
    if (rc) return rc;
    // slope of the imposed body force in the x-z plane, density ratio of
    // the particles to the liquid (reference density 1), |g| the magnitude
    // of the body acceleration (Section 4.2, Table 2)
    const double tanpsi = d.gzd != 0.0 ? d.gxd / std::fabs(d.gzd) : 0.0;
    const double s1 = s->p.rho_p - 1.0;
    const double gm = std::sqrt(d.gxd * d.gxd + d.gyd * d.gyd + d.gzd * d.gzd);
    out[0] = dep[0];
    out[1] = tanpsi;
    out[2] = s1 != 0.0 ? dep[0] * tanpsi / (d50 * s1) : 0.0;
    out[3] = red[6];
    out[4] = (s1 > 0.0 && gm > 0.0) ? red[6] / std::sqrt(s1 * gm * d50 * d50 * d50) : 0.0;
    out[5] = dep[1];
    return FSLBM_OK;
}

int fslbm_bed_spectrum(const double* h, int64_t nt, int64_t nx, double dx, double dt, double* psd, double peak[4],
                       void* cuda_stream) {
    if (!h || !psd || !peak || nt < 2 || nx < 2 || nt > 65535 || nx > (1 << 20)) return FSLBM_EINVAL;
    if (!(dx > 0.0) || !(dt > 0.0) || !std::isfinite(dx) || !std::isfinite(dt)) return FSLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    // scratch: twiddles (nx + nt complex), the x-transformed series (nt nx
    // complex), the mean, and the peak (value, l, j)
    const size_t work_doubles = 2 * ((size_t)nx + nt + (size_t)nt * nx) + 4;
    double* work = nullptr;
    if (cudaMalloc(&work, work_doubles * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return FSLBM_ENOMEM;
    }
    double* peak3 = work + work_doubles - 3;
    cudaGetLastError();
    launch_bed_spectrum(h, (int)nt, (int)nx, psd, work, peak3, st);
    double pk[3] = {0.0, 0.0, 0.0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(pk, peak3, sizeof(pk), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(work);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return FSLBM_EDEVICE;
    }
    // the transform kernel is exp(-2 pi i (j x / nx + l t / nt)): a bedform
    // moving toward +x at wavenumber j > 0 has frequency index l < 0
    const long long l = (long long)pk[1], j = (long long)pk[2];
    const long long ls = l <= nt / 2 ? l : l - nt;
    const double lam = (double)nx * dx / (double)j;
    peak[0] = lam;
    peak[1] = ls == 0 ? INFINITY : (double)nt * dt / (double)(ls < 0 ? -ls : ls);
    peak[2] = ls == 0 ? 0.0 : (ls < 0 ? 1.0 : -1.0) * lam / peak[1];
    peak[3] = 2.0 * std::sqrt(pk[0] / ((double)nt * (double)nx));
    return FSLBM_OK;
}

int fslbm_set_wait_limit(fslbm* s, int64_t polls) {
    if (!s || polls < 0 || polls > WAIT_LIMIT_DEFAULT) return FSLBM_EINVAL;
    s->d.wait_limit = (int)polls;
    s->graph_dirty = true;
    return FSLBM_OK;
}

int fslbm_set_normal_model(fslbm* s, const uint16_t* w, int64_t n_params) {
    if (!s) return FSLBM_EINVAL;
    if (s->host_err) return s->host_err;
    Dev& d = s->d;
    MlpBf16 h;
    std::vector<__nv_bfloat16> w1m;
    std::vector<MlpFrag> frag;
    if (!w) {
        if (n_params != 0) return FSLBM_EINVAL;
        d.mlp = nullptr;
        d.mlp_stats = nullptr;
        d.mlp_frag = nullptr;
        s->p.normal_model = 0;
    } else {
        if (n_params != MLP_NPARAM) return FSLBM_EINVAL;
        bool ok = true;
        if (!s->mlp_dev) s->mlp_dev = dalloc<MlpBf16>(s, 1, ok);
        if (!s->mlp_stats) s->mlp_stats = dalloc<unsigned long long>(s, 2, ok);
        if (!s->mlp_frag_dev) s->mlp_frag_dev = dalloc<MlpFrag>(s, 1, ok);
        if (!ok) return FSLBM_ENOMEM;
        mlp_from_bf16_host(w, h);
        w1m.resize(3 * MLP_H * 32);
        mlp_mirror_w1_host(w, w1m.data());
        frag.resize(1);
        mlp_frag_host(h, w1m.data(), frag[0]);
        cudaMemcpyAsync(s->mlp_dev, &h, sizeof(h), cudaMemcpyHostToDevice, s->st);
        cudaMemcpyAsync(s->mlp_frag_dev, frag.data(), sizeof(MlpFrag), cudaMemcpyHostToDevice, s->st);
        cudaMemsetAsync(s->mlp_stats, 0, 2 * sizeof(unsigned long long), s->st);
        d.mlp = s->mlp_dev;
        d.mlp_stats = s->mlp_stats;
        d.mlp_frag = s->mlp_frag_dev;
        s->p.normal_model = 1;
    }
    s->graph_dirty = true;
    launch_normals(d, d.nrm, s->st);
    return sync_check(s);   // h and frag stay alive until the copies have completed
}

int fslbm_set_normal_mirror(fslbm* s, int32_t on) {
    if (!s || (on != 0 && on != 1)) return FSLBM_EINVAL;
    if (s->host_err) return s->host_err;
    s->d.mlp_mirror = on;
    s->graph_dirty = true;
    if (s->d.mlp) launch_normals(s->d, s->d.nrm, s->st);
    return sync_check(s);
}

int fslbm_normal_stats(fslbm* s, uint64_t out[2]) {
    if (!s || !out) return FSLBM_EINVAL;
    out[0] = out[1] = 0;
    if (!s->d.mlp_stats) return FSLBM_OK;
    unsigned long long h[2] = {0, 0};
    cudaMemcpyAsync(h, s->d.mlp_stats, sizeof(h), cudaMemcpyDeviceToHost, s->st);
    const int rc = sync_check(s);
    out[0] = h[0];
    out[1] = h[1];
    return rc;
}

int fslbm_log_stencils(fslbm* s, int64_t capacity, float* fill, float* target, float* fd, int32_t* cells,
                       int64_t* found) {
    if (!s || !found || capacity < 0 || (capacity > 0 && (!fill || !target))) return FSLBM_EINVAL;
    *found = 0;
    if (s->host_err) return s->host_err;
    // the counter lives in the reduction's output block (8 doubles), whose
    // values no caller reads across this call
    unsigned long long* dfound = reinterpret_cast<unsigned long long*>(s->red);
    launch_log_stencils(s->d, capacity, fill, target, fd, cells, dfound, s->st);
    unsigned long long h = 0;
    cudaMemcpyAsync(&h, dfound, sizeof(h), cudaMemcpyDeviceToHost, s->st);
    const int rc = sync_check(s);
    if (rc) return rc;
    *found = (int64_t)h;
    return launch_check(s);
}

void fslbm_destroy(fslbm* s) {
    if (!s) return;
    cudaStreamSynchronize(s->st);
    if (s->side) {
        cudaStreamSynchronize(s->side);
        cudaStreamDestroy(s->side);
    }
    if (s->ev_fork) cudaEventDestroy(s->ev_fork);
    if (s->ev_join) cudaEventDestroy(s->ev_join);
    for (int k = 0; k < 2; ++k) {
        drop_graph(s, k);
        if (s->ev_cap[k]) cudaEventDestroy(s->ev_cap[k]);
    }
    for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
    for (void* p : s->allocs) cudaFree(p);
    delete s;
}

}  // extern "C"
