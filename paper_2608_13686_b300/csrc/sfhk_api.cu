// sfhk_api.cu -- the C ABI of libsfhk (include/sfhk.h): handles, device-memory
// budget, argument checking and the launch sequences of each entry point.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sfhk_device.cuh"
#include "sfhk_internal.h"


namespace sfhk {

std::atomic<unsigned long long> g_launches{0};

int Ctx::alloc(DeviceBuf& b, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    if (budget != 0 && used.load() + bytes > budget) return SFHK_E_NOMEM;
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SFHK_E_NOMEM;
    }
    b.p = p;
    b.bytes = bytes;
    used += bytes;
    return SFHK_OK;
}

void Ctx::release(DeviceBuf& b)
{
    if (b.p) {
        cudaFree(b.p);
        used -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
}

namespace {

constexpr double kPi = 3.14159265358979323846;

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

// 1 / sqrt(<phi|phi>) for phi = sum_c sum_k coef_k g_k(r - R_c), the
// centres at z_c = s_c R/2 on the axis n.  Two primitives on centres A, B
// multiply to e^{-ab/p (z_A - z_B)^2} e^{-p |r - P|^2} (p = a + b, P on the
// axis at z_P = (a z_A + b z_B)/p), whose integral is S0 = (pi/p)^{3/2}
// e^{-ab/p (z_A - z_B)^2}.  Writing n.(r - A) = n.(r - P) + (z_P - z_A) and
// using int n.(r-P) e^{-p|r-P|^2} = 0, int [n.(r-P)]^2 e^{-p|r-P|^2} =
// S0 / (2p): an s-s pair gives S0, an s-p pair s_B (z_P - z_B) S0 and a p-p
// pair s_A s_B [(z_P - z_A)(z_P - z_B) + 1/(2p)] S0.  A pi p-type factor
// m.(r - A) has m perpendicular to the axis, so m.(P - A) = 0: it overlaps
// only another pi primitive (m.m = 1), by S0 / (2p).
double orbital_norm(const sfhk_target_desc& d)
{
    double s = 0.0;
    for (int c1 = 0; c1 < 2; ++c1)
        for (int c2 = 0; c2 < 2; ++c2) {
            const double s1 = c1 == 0 ? 1.0 : -1.0, s2 = c2 == 0 ? 1.0 : -1.0;
            const double z1 = 0.5 * s1 * d.R, z2 = 0.5 * s2 * d.R;
            for (int k1 = 0; k1 < d.n_prim; ++k1)
                for (int k2 = 0; k2 < d.n_prim; ++k2) {
                    const double a = d.prim_exp[k1], b = d.prim_exp[k2], pab = a + b;
                    const double zP = (a * z1 + b * z2) / pab;
                    const double S0 = std::pow(kPi / pab, 1.5) *
                                      std::exp(-a * b / pab * (z1 - z2) * (z1 - z2));
                    const int t1 = d.prim_kind[k1], t2 = d.prim_kind[k2];
                    const bool p1 = t1 == SFHK_PRIM_P_SIGMA, p2 = t2 == SFHK_PRIM_P_SIGMA;
                    double ang = 1.0;
                    if (t1 == SFHK_PRIM_P_PI || t2 == SFHK_PRIM_P_PI)
                        ang = (t1 == t2) ? 0.5 / pab : 0.0;
                    else if (p1 && p2) ang = s1 * s2 * ((zP - z1) * (zP - z2) + 0.5 / pab);
                    else if (p1) ang = s1 * (zP - z1);
                    else if (p2) ang = s2 * (zP - z2);
                    s += d.prim_coef[k1] * d.prim_coef[k2] * ang * S0;
                }
        }
    return s > 0.0 ? 1.0 / std::sqrt(s) : INFINITY;
}

// Recombination constants per primitive (a its exponent, b = gamma/2,
// c = a + b): K1 = -ab/c, K2 = -1/(4c), K3 = -a/c and
// K4 = N coef (gamma/pi)^{3/4} (pi/c)^{3/2} a/c; a sigma p-type primitive
// adds P1 = b/c, P2 = 1/(2c), P3 = gamma/(2a).
// 1 / sqrt(<phi|phi>) of a polyatomic orbital phi = sum_k coef_k f_k(r - A_k)
// e^{-a_k |r - A_k|^2} (molecular frame; f = 1, or u_k.(r - A_k) with u_k the
// unit p direction).  A pair of primitives multiplies to S0 e^{-p |r - P|^2},
// p = a + b, P = (a A + b B)/p, S0 = (pi/p)^{3/2} e^{-ab/p |A - B|^2} after
// integration; with y = r - P a p factor is u.y + u.(P - A), whose odd part
// integrates to zero and whose square part gives u_1.u_2 / (2p).
double poly_norm(const sfhk_target_desc& d, const double (*udir)[3])
{
    double s = 0.0;
    for (int i = 0; i < d.n_prim; ++i)
        for (int j = 0; j < d.n_prim; ++j) {
            const double* A = d.centre_pos[d.prim_centre[i]];
            const double* B = d.centre_pos[d.prim_centre[j]];
            const double a = d.prim_exp[i], b = d.prim_exp[j], pab = a + b;
            double AB2 = 0.0, ai = 0.0, aj = 0.0, uu = 0.0;
            for (int x = 0; x < 3; ++x) {
                const double P = (a * A[x] + b * B[x]) / pab;
                AB2 += (A[x] - B[x]) * (A[x] - B[x]);
                ai += udir[i][x] * (P - A[x]);
                aj += udir[j][x] * (P - B[x]);
                uu += udir[i][x] * udir[j][x];
            }
            const bool pi = d.prim_kind[i] == SFHK_PRIM_P_DIR, pj = d.prim_kind[j] == SFHK_PRIM_P_DIR;
            const double ang = (pi && pj) ? ai * aj + 0.5 * uu / pab : pi ? ai : pj ? aj : 1.0;
            s += d.prim_coef[i] * d.prim_coef[j] * ang * std::pow(kPi / pab, 1.5) *
                 std::exp(-a * b / pab * AB2);
        }
    return s > 0.0 ? 1.0 / std::sqrt(s) : INFINITY;
}

void fill_recomb(const DevTarget& T, double gamma, DevRecomb& R)
{
    const double b = 0.5 * gamma;
    R.has_p = 0;
    R.cchi = std::cos(T.pi_azimuth);
    R.schi = std::sin(T.pi_azimuth);
    for (int k = 0; k < SFHK_MAX_PRIM; ++k) {
        R.kind[k] = 0;
        if (k >= T.n_prim) {
            R.K1[k] = R.K2[k] = R.K3[k] = R.K4[k] = 0.0;
            R.P1[k] = R.P2[k] = R.P3[k] = 0.0;
        } else {
            const double a = T.pexp[k], c = a + b;
            R.K1[k] = -a * b / c;
            R.K2[k] = -1.0 / (4.0 * c);
            R.K3[k] = -a / c;
            R.K4[k] = T.norm * T.pcoef[k] * std::pow(gamma / kPi, 0.75) * std::pow(kPi / c, 1.5) *
                      (a / c);
            R.kind[k] = T.pkind[k];
            R.P1[k] = b / c;
            R.P2[k] = 0.5 / c;
            R.P3[k] = gamma / (2.0 * a);
            if (T.pkind[k] == 1 || T.pkind[k] == 2) R.has_p |= T.pkind[k];   // bit 0 sigma, bit 1 pi
        }
        R.K1f[k] = (float)R.K1[k];
        R.K2f[k] = (float)R.K2[k];
        R.K3f[k] = (float)R.K3[k];
        R.K4f[k] = (float)R.K4[k];
        R.P1f[k] = (float)R.P1[k];
        R.P2f[k] = (float)R.P2[k];
        R.P3f[k] = (float)R.P3[k];
    }
}

// Table rows of the polyatomic kernel for a set of ensembles launched
// together: 0 for diatomic targets, else the largest n_slots; SFHK_E_INVAL
// when the set mixes the two.  nc (may be null): the centre count the
// polyatomic targets share, 0 when they differ.
int poly_slots(sfhk_ensemble* const* ens, int n_ens, int* slots, int* nc)
{
    int np = 0, mx = 0, common = -1;
    for (int i = 0; i < n_ens; ++i) {
        const DevTarget& T = ens[i]->tgt->dev;
        if (T.kind == SFHK_POT_POLYATOMIC) {
            ++np;
            mx = std::max(mx, std::max(1, T.n_slots));
            common = (common < 0 || common == T.n_centres) ? T.n_centres : 0;
        }
    }
    if (np != 0 && np != n_ens) return SFHK_E_INVAL;
    *slots = mx;
    if (nc) *nc = common > 0 ? common : 0;
    return SFHK_OK;
}

int set_device(int dev)
{
    SFHK_CUDA_TRY(cudaSetDevice(dev));
    return SFHK_OK;
}

// buffers every ensemble owns, allocated once
int ensemble_alloc(sfhk_ensemble* e, long long n, int nt)
{
    Ctx* c = e->ctx;
    const long long n_items = (n + kWarp - 1) / kWarp;
    int rc;
    if ((rc = c->alloc(e->soa, sizeof(double) * kSoaFields * (size_t)n))) return rc;
    if ((rc = c->alloc(e->n0, sizeof(int) * (size_t)n))) return rc;
    if ((rc = c->alloc(e->perm, sizeof(int) * (size_t)n))) return rc;
    if ((rc = c->alloc(e->items, sizeof(WorkItem) * (size_t)n_items))) return rc;
    if ((rc = c->alloc(e->ph, sizeof(double2) * nt))) return rc;
    if ((rc = c->alloc(e->phf, sizeof(float2) * nt))) return rc;
    if ((rc = c->alloc(e->vz, sizeof(double) * nt))) return rc;
    if ((rc = c->alloc(e->counters, sizeof(unsigned long long) * 8))) return rc;
    if ((rc = c->alloc(e->cdf, sizeof(double) * cdf_doubles(nt)))) return rc;
    if ((rc = c->alloc(e->hist, sizeof(int) * nt))) return rc;
    if ((rc = c->alloc(e->inst, sizeof(DevInstance)))) return rc;
    if ((rc = c->alloc(e->qctr, sizeof(unsigned int) * 4))) return rc;
    e->n_items = (int)n_items;
    SFHK_CUDA_TRY(cudaEventCreate(&e->ev_start));
    SFHK_CUDA_TRY(cudaEventCreate(&e->ev_stop));
    SFHK_CUDA_TRY(cudaEventCreateWithFlags(&e->ev_done, cudaEventDisableTiming));
    return SFHK_OK;
}

void ensemble_free(sfhk_ensemble* e)
{
    if (!e) return;
    Ctx* c = e->ctx;
    for (DeviceBuf* b : {&e->soa, &e->n0, &e->perm, &e->items, &e->ph, &e->phf, &e->vz,
                         &e->dump, &e->counters, &e->cdf, &e->hist, &e->inst, &e->qctr,
                         &e->returns, &e->pilot})
        c->release(*b);
    if (e->ev_start) cudaEventDestroy(e->ev_start);
    if (e->ev_stop) cudaEventDestroy(e->ev_stop);
    if (e->ev_done) cudaEventDestroy(e->ev_done);
    delete e;
}

// sort by birth index, build the warp work items, the phase table
int ensemble_finish(sfhk_ensemble* e, cudaStream_t s)
{
    int rc = launch_counting_sort((const int*)e->n0.p, e->n, e->pulse->nt, (int*)e->perm.p,
                                  (int*)e->hist.p, s);
    if (rc) return rc;
    rc = launch_build_items((const int*)e->perm.p, (const int*)e->n0.p, e->n, 0,
                            (WorkItem*)e->items.p, s);
    if (rc) return rc;
    return launch_phase_table(*e->pulse, e->tgt->desc.Ip, (double2*)e->ph.p, (float2*)e->phf.p, s);
}

}  // namespace

DevInstance make_instance(sfhk_ensemble* e, const sfhk_run_opts& o)
{
    DevInstance I;
    std::memset(&I, 0, sizeof I);
    I.tgt = e->tgt->dev;
    fill_recomb(I.tgt, o.gamma, I.rec);
    I.Eh = (const double*)e->pulse->Eh.p;
    I.Ehf = (const float*)e->pulse->Ehf.p;
    I.ph = (const double2*)e->ph.p;
    I.phf = (const float2*)e->phf.p;
    I.soa = (const double*)e->soa.p;
    I.perm = (const int*)e->perm.p;
    I.n0 = (const int*)e->n0.p;
    I.vz = (double*)e->vz.p;
    I.dump = o.dump_final ? (double*)e->dump.p : nullptr;
    I.returns = o.record_returns ? (double*)e->returns.p : nullptr;
    I.ret_out = o.return_r_out;
    I.ret_in = o.return_r_in;
    I.counters = (unsigned long long*)e->counters.p;
    I.n = e->n;
    I.nt = e->pulse->nt;
    I.dt = e->pulse->dt;
    I.t_origin = e->pulse->t_origin;
    I.scale = -2.0 / (e->n_norm > 0.0 ? e->n_norm : (double)e->n);
    I.gamma = o.gamma;
    I.inv_gamma = 1.0 / o.gamma;
    I.cutoff2 = o.prefactor_cutoff > 0.0 ? o.prefactor_cutoff * o.prefactor_cutoff : 0.0;
    I.stab_cut = o.stability_cutoff > 0.0 ? o.stability_cutoff : 0.0;
    // tapered stability filter: stop at r m0, weight by the taper above m0
    const bool taper = I.stab_cut > 0.0 && o.stability_taper > 1.0;
    I.stab_hi = taper ? o.stability_taper * I.stab_cut : 0.0;
    I.inv_log_taper = taper ? 1.0 / std::log(o.stability_taper) : 0.0;
    I.done_items = nullptr;
    I.cancel = nullptr;
    return I;
}

namespace {

int check_opts(const sfhk_run_opts* o)
{
    if (!o) return SFHK_E_INVAL;
    if (o->precision != SFHK_FP64 && o->precision != SFHK_MIXED) return SFHK_E_INVAL;
    if (!(o->gamma > 0.0) || !std::isfinite(o->gamma)) return SFHK_E_INVAL;
    if (o->prefactor_cutoff < 0.0 || o->stability_cutoff < 0.0) return SFHK_E_INVAL;
    if (!(o->stability_taper == 0.0 || o->stability_taper > 1.0) ||
        !std::isfinite(o->stability_taper))
        return SFHK_E_INVAL;
    if (o->block_threads < 0 || o->block_threads > 128 || o->block_threads % 32) return SFHK_E_INVAL;
    if (o->blocks_per_sm < 0) return SFHK_E_INVAL;
    if (o->kernel_variant < 0 || o->kernel_variant > kPropVariants) return SFHK_E_INVAL;
    if (o->record_returns && !(o->return_r_in > 0.0 && o->return_r_out > o->return_r_in &&
                               std::isfinite(o->return_r_out)))
        return SFHK_E_INVAL;
    if (o->check_nonfinite != 0 && o->check_nonfinite != 1) return SFHK_E_INVAL;
    return SFHK_OK;
}

// the non-finite limit that sfhk_dipole / sfhk_stats_get apply to the
// ensemble's last propagation
void set_nonfinite_limit(sfhk_ensemble* e, const sfhk_run_opts& o)
{
    e->check_nonfinite = o.check_nonfinite != 0;
    e->max_nonfinite = (unsigned long long)o.max_nonfinite;
}

}  // namespace

// prepare one ensemble for a launch: zero outputs, dump buffer
int prepare_outputs(sfhk_ensemble* e, const sfhk_run_opts& o, cudaStream_t s)
{
    Ctx* c = e->ctx;
    if (o.dump_final && !e->dump.p) {
        int rc = c->alloc(e->dump, sizeof(double) * kFinalFields * (size_t)e->n);
        if (rc) return rc;
    }
    if (o.record_returns && !e->returns.p) {
        int rc = c->alloc(e->returns, sizeof(double) * 2 * (size_t)e->n);
        if (rc) return rc;
    }
    e->returns_kept = o.record_returns != 0;
    SFHK_CUDA_TRY(cudaMemsetAsync(e->vz.p, 0, sizeof(double) * e->pulse->nt, s));
    SFHK_CUDA_TRY(cudaMemsetAsync(e->counters.p, 0, sizeof(unsigned long long) * 3, s));
    SFHK_CUDA_TRY(cudaMemsetAsync((unsigned long long*)e->counters.p + 4, 0,
                                  sizeof(unsigned long long) * 2, s));
    e->dumped = o.dump_final != 0;
    return SFHK_OK;
}

namespace {

// the launch shape: the run options' where set, else the context's tuned
// shape for the precision and the launch's integrator form (fixed_form)
void shape(Ctx* c, const sfhk_run_opts& o, int form, int* bt, int* var, int* bps)
{
    const int* t = c->tuned[o.precision][form];
    *bt = o.block_threads > 0 ? o.block_threads : t[0];
    *var = o.kernel_variant > 0 ? o.kernel_variant - 1 : t[1];
    *bps = o.blocks_per_sm > 0 ? o.blocks_per_sm : t[2];
}

}  // namespace
}  // namespace sfhk

using namespace sfhk;

extern "C" {

const char* sfhk_strerror(int code)
{
    switch (code) {
    case SFHK_OK: return "ok";
    case SFHK_E_INVAL: return "invalid argument";
    case SFHK_E_NOMEM: return "device memory budget or allocation exceeded";
    case SFHK_E_CUDA: return "CUDA error or no compute-capability-10.3 device";
    case SFHK_E_TIMEOUT: return "bounded wait expired";
    case SFHK_E_NUMERIC: return "too many non-finite trajectories";
    case SFHK_E_BUSY: return "result not ready";
    case SFHK_E_NOTFOUND: return "unknown request id";
    default: return "unknown error";
    }
}

int sfhk_create(sfhk_ctx** out, int device, size_t budget)
{
    if (!out) return SFHK_E_INVAL;
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
        cudaGetLastError();
        return SFHK_E_CUDA;
    }
    cudaDeviceProp prop;
    SFHK_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3) return SFHK_E_CUDA;
    SFHK_CUDA_TRY(cudaSetDevice(device));
    int rc = configure_kernels();
    if (rc) return rc;
    sfhk_ctx* c = new (std::nothrow) sfhk_ctx;
    if (!c) return SFHK_E_NOMEM;
    c->device = device;
    c->sm_count = prop.multiProcessorCount;
    c->budget = budget;
    *out = c;
    return SFHK_OK;
}

int sfhk_destroy(sfhk_ctx* c)
{
    if (!c) return SFHK_E_INVAL;
    delete c;
    return SFHK_OK;
}

int sfhk_mem_used(const sfhk_ctx* c, size_t* bytes)
{
    if (!c || !bytes) return SFHK_E_INVAL;
    *bytes = c->used.load();
    return SFHK_OK;
}

int sfhk_create_target(sfhk_ctx* c, const sfhk_target_desc* d, sfhk_target** out)
{
    if (!c || !d || !out) return SFHK_E_INVAL;
    if (d->kind != SFHK_POT_MOLECULE && d->kind != SFHK_POT_HARMONIC &&
        d->kind != SFHK_POT_POLYATOMIC)
        return SFHK_E_INVAL;
    if (d->n_prim < 1 || d->n_prim > SFHK_MAX_PRIM) return SFHK_E_INVAL;
    if (d->ionization != SFHK_IONIZE_SFA && d->ionization != SFHK_IONIZE_MODIFIED)
        return SFHK_E_INVAL;
    if ((d->sampling != SFHK_SAMPLE_PROPOSAL && d->sampling != SFHK_SAMPLE_ABS_AMPLITUDE) ||
        !std::isfinite(d->sampling_factor))
        return SFHK_E_INVAL;
    for (int k = 0; k < d->n_prim; ++k)
        if (!(d->prim_exp[k] > 0.0) || !std::isfinite(d->prim_coef[k]) ||
            d->prim_kind[k] < SFHK_PRIM_S || d->prim_kind[k] > SFHK_PRIM_P_DIR)
            return SFHK_E_INVAL;
    if (!std::isfinite(d->pi_azimuth)) return SFHK_E_INVAL;
    const bool poly = d->kind == SFHK_POT_POLYATOMIC;
    // p-type along a given direction on polyatomic targets only; sigma and
    // pi p-type on diatomic targets only
    for (int k = 0; k < d->n_prim; ++k)
        if (d->prim_kind[k] != SFHK_PRIM_S && (d->prim_kind[k] == SFHK_PRIM_P_DIR) != poly)
            return SFHK_E_INVAL;
    if (poly) {
        if (d->n_centres < 1 || d->n_centres > SFHK_MAX_CENTRES) return SFHK_E_INVAL;
        if (d->ionization != SFHK_IONIZE_SFA) return SFHK_E_INVAL;
        for (int c = 0; c < d->n_centres; ++c) {
            for (int a = 0; a < 3; ++a)
                if (!std::isfinite(d->centre_pos[c][a])) return SFHK_E_INVAL;
            if (!std::isfinite(d->centre_Z_inf[c]) || !std::isfinite(d->centre_Z0[c]) ||
                !(d->centre_alpha[c] >= 0.0) || !std::isfinite(d->centre_alpha[c]))
                return SFHK_E_INVAL;
        }
        for (int k = 0; k < d->n_prim; ++k) {
            if (d->prim_centre[k] < 0 || d->prim_centre[k] >= d->n_centres) return SFHK_E_INVAL;
            if (d->prim_kind[k] == SFHK_PRIM_P_DIR) {
                const double* u = d->prim_dir[k];
                const double l2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
                if (!(l2 > 0.0) || !std::isfinite(l2)) return SFHK_E_INVAL;
            }
        }
    }
    if (d->soft_a < 0.0 || d->R < 0.0 || d->alpha < 0.0 || !std::isfinite(d->Ip)) return SFHK_E_INVAL;
    if (d->kind == SFHK_POT_MOLECULE && d->soft_a == 0.0 && d->Z_inf == 0.0 && d->Z0 == 0.0)
        ;  // a field-free "molecule" is allowed
    sfhk_target* t = new (std::nothrow) sfhk_target;
    if (!t) return SFHK_E_NOMEM;
    t->ctx = c;
    t->desc = *d;
    for (int k = d->n_prim; k < SFHK_MAX_PRIM; ++k) {
        t->desc.prim_exp[k] = t->desc.prim_coef[k] = 0.0;
        t->desc.prim_kind[k] = SFHK_PRIM_S;
    }
    DevTarget& T = t->dev;
    std::memset(&T, 0, sizeof T);
    T.kind = d->kind;
    T.n_prim = d->n_prim;
    T.half_R = 0.5 * d->R;
    T.Zinf = d->Z_inf;
    T.dZ = d->Z0 - d->Z_inf;
    T.screened = T.dZ != 0.0;
    T.alpha = d->alpha;
    T.a2 = d->soft_a * d->soft_a;
    T.Ip = d->Ip;
    T.w2 = d->ho_omega * d->ho_omega;
    for (int k = 0; k < SFHK_MAX_PRIM; ++k) {
        T.pexp[k] = t->desc.prim_exp[k];
        T.pcoef[k] = t->desc.prim_coef[k];
        T.pkind[k] = t->desc.prim_kind[k];
    }
    T.pi_azimuth = d->pi_azimuth;
    if (poly) {
        T.n_centres = d->n_centres;
        bool any_p = false;
        for (int c = 0; c < d->n_centres; ++c) {
            for (int a = 0; a < 3; ++a) T.cpos[c][a] = d->centre_pos[c][a];
            T.cZinf[c] = d->centre_Z_inf[c];
            T.cdZ[c] = d->centre_Z0[c] - d->centre_Z_inf[c];
            T.calpha[c] = d->centre_alpha[c];
            T.cq_f[c] = make_float4((float)T.cZinf[c], (float)T.cdZ[c], (float)T.calpha[c], 0.0f);
        }
        for (int c = 0; c + 1 < d->n_centres; c += 2) {
            const float4 a = T.cq_f[c], b = T.cq_f[c + 1];
            T.cq2_f[c / 2][0] = make_float4(a.x, b.x, a.y, b.y);
            T.cq2_f[c / 2][1] = make_float4(a.z, b.z, 0.0f, 0.0f);
        }
        for (int k = 0; k < d->n_prim; ++k) {
            T.pcentre[k] = d->prim_centre[k];
            if (d->prim_kind[k] == SFHK_PRIM_P_DIR) {
                const double* u = d->prim_dir[k];
                const double l = std::sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
                for (int a = 0; a < 3; ++a) T.pdir[k][a] = u[a] / l;
                any_p = true;
            }
        }
        T.n_slots = T.n_centres + (any_p ? d->n_prim : 0);
    }
    T.norm = poly ? poly_norm(t->desc, T.pdir) : orbital_norm(t->desc);
    if (!std::isfinite(T.norm)) {
        delete t;
        return SFHK_E_INVAL;
    }
    *out = t;
    return SFHK_OK;
}

int sfhk_destroy_target(sfhk_target* t)
{
    if (!t) return SFHK_E_INVAL;
    delete t;
    return SFHK_OK;
}

int sfhk_set_pulse(sfhk_ctx* c, const sfhk_pulse_desc* d, sfhk_pulse** out)
{
    if (!c || !d || !out) return SFHK_E_INVAL;
    if (!(d->lambda_nm > 0.0) || !(d->dt > 0.0) || !(d->n_cycles >= 1.5) ||
        !(d->intensity_Wcm2 >= 0.0) || !std::isfinite(d->cep))
        return SFHK_E_INVAL;
    const double omega = 45.5633525 / d->lambda_nm;
    const double Tp = d->n_cycles * 2.0 * kPi / omega;
    const double steps = std::floor(Tp / d->dt * (1.0 + 1e-12));
    if (!(steps >= 1.0) || steps > double(1 << 26)) return SFHK_E_INVAL;
    int rc = set_device(c->device);
    if (rc) return rc;
    sfhk_pulse* p = new (std::nothrow) sfhk_pulse;
    if (!p) return SFHK_E_NOMEM;
    p->ctx = c;
    p->desc = *d;
    p->omega = omega;
    p->E0 = std::sqrt(d->intensity_Wcm2 / 3.50944758e16);
    p->Tp = Tp;
    p->t_origin = -0.5 * Tp;
    p->dt = d->dt;
    p->nt = (int)steps + 1;
    const int m = 2 * p->nt - 1;
    if ((rc = c->alloc(p->Eh, sizeof(double) * m)) || (rc = c->alloc(p->Ehf, sizeof(float) * m))) {
        c->release(p->Eh);
        delete p;
        return rc;
    }
    rc = launch_field_table(*p, (double*)p->Eh.p, (float*)p->Ehf.p, 0);
    if (!rc && cudaStreamSynchronize(0) != cudaSuccess) rc = SFHK_E_CUDA;
    if (rc) {
        c->release(p->Eh);
        c->release(p->Ehf);
        delete p;
        return rc;
    }
    *out = p;
    return SFHK_OK;
}

int sfhk_destroy_pulse(sfhk_pulse* p)
{
    if (!p) return SFHK_E_INVAL;
    p->ctx->release(p->Eh);
    p->ctx->release(p->Ehf);
    delete p;
    return SFHK_OK;
}

int sfhk_pulse_grid(const sfhk_pulse* p, int* nt, double* t_origin, double* dt, double* Tp)
{
    if (!p) return SFHK_E_INVAL;
    if (nt) *nt = p->nt;
    if (t_origin) *t_origin = p->t_origin;
    if (dt) *dt = p->dt;
    if (Tp) *Tp = p->Tp;
    return SFHK_OK;
}

int sfhk_sample_initial(sfhk_ctx* c, const sfhk_target* t, const sfhk_pulse* p,
                        const sfhk_align_desc* al, uint64_t n_traj, uint64_t seed,
                        uint32_t instance, sfhk_ensemble** out, void* stream)
{
    if (!c || !t || !p || !al || !out) return SFHK_E_INVAL;
    if (n_traj == 0 || n_traj > 2147483647ull) return SFHK_E_INVAL;
    if (!(t->desc.Ip > 0.0) || !(p->E0 > 0.0)) return SFHK_E_INVAL;
    if (!align_valid(*al)) return SFHK_E_INVAL;
    int rc = set_device(c->device);
    if (rc) return rc;
    sfhk_ensemble* e = new (std::nothrow) sfhk_ensemble;
    if (!e) return SFHK_E_NOMEM;
    e->ctx = c;
    e->tgt = t;
    e->pulse = p;
    e->n = (long long)n_traj;
    e->n_norm = (double)n_traj;
    if ((rc = ensemble_alloc(e, e->n, p->nt)) ||
        (t->desc.sampling == SFHK_SAMPLE_ABS_AMPLITUDE &&
         (rc = c->alloc(e->pilot, sizeof(double) * sample_pilot_doubles())))) {
        ensemble_free(e);
        return rc;
    }
    cudaStream_t s = as_stream(stream);
    unsigned long long* cnt = (unsigned long long*)e->counters.p;
    if (cudaMemsetAsync(cnt, 0, sizeof(unsigned long long) * 8, s) != cudaSuccess) rc = SFHK_E_CUDA;
    if (!rc) rc = launch_adk_cdf(*p, t->desc.Ip, (double*)e->cdf.p, s);
    if (!rc)
        rc = launch_sample(*t, *p, *al, e->n, seed, instance, (const double*)e->cdf.p,
                           (double*)e->soa.p, (int*)e->n0.p, cnt + 3, (double*)e->pilot.p, s);
    if (!rc) rc = ensemble_finish(e, s);
    e->sampled = true;
    if (rc) {
        cudaStreamSynchronize(s);
        ensemble_free(e);
        return rc;
    }
    *out = e;
    return SFHK_OK;
}

int sfhk_sample_into(sfhk_ctx* c, sfhk_ensemble* e, const sfhk_align_desc* al, uint64_t seed,
                     uint32_t instance, void* stream)
{
    if (!c || !e || !al || e->ctx != c || !e->sampled) return SFHK_E_INVAL;
    if (!align_valid(*al)) return SFHK_E_INVAL;
    int rc = set_device(c->device);
    if (rc) return rc;
    cudaStream_t s = as_stream(stream);
    unsigned long long* cnt = (unsigned long long*)e->counters.p;
    SFHK_CUDA_TRY(cudaMemsetAsync(cnt + 3, 0, sizeof(unsigned long long), s));
    rc = launch_sample(*e->tgt, *e->pulse, *al, e->n, seed, instance, (const double*)e->cdf.p,
                       (double*)e->soa.p, (int*)e->n0.p, cnt + 3, (double*)e->pilot.p, s);
    if (rc) return rc;
    rc = launch_counting_sort((const int*)e->n0.p, e->n, e->pulse->nt, (int*)e->perm.p,
                              (int*)e->hist.p, s);
    if (rc) return rc;
    rc = launch_build_items((const int*)e->perm.p, (const int*)e->n0.p, e->n, 0,
                            (WorkItem*)e->items.p, s);
    e->have_result = false;
    return rc;
}

int sfhk_launch_count(uint64_t* out)
{
    if (!out) return SFHK_E_INVAL;
    *out = g_launches.load();
    return SFHK_OK;
}

int sfhk_load_ensemble(sfhk_ctx* c, const sfhk_target* t, const sfhk_pulse* p,
                       const double* soa_host, uint64_t n_traj, double n_norm,
                       sfhk_ensemble** out)
{
    if (!c || !t || !p || !soa_host || !out) return SFHK_E_INVAL;
    if (n_traj == 0 || n_traj > 2147483647ull || n_norm < 0.0) return SFHK_E_INVAL;
    const long long n = (long long)n_traj;
    for (long long j = 0; j < n; ++j) {
        const double m = soa_host[j];
        if (!(m >= 0.0) || m > double(p->nt - 1) || m != std::floor(m)) return SFHK_E_INVAL;
    }
    for (long long i = n; i < (long long)kSoaFields * n; ++i)
        if (!std::isfinite(soa_host[i])) return SFHK_E_INVAL;
    int rc = set_device(c->device);
    if (rc) return rc;
    sfhk_ensemble* e = new (std::nothrow) sfhk_ensemble;
    if (!e) return SFHK_E_NOMEM;
    e->ctx = c;
    e->tgt = t;
    e->pulse = p;
    e->n = n;
    e->n_norm = n_norm > 0.0 ? n_norm : (double)n;
    if ((rc = ensemble_alloc(e, n, p->nt))) {
        ensemble_free(e);
        return rc;
    }
    if (cudaMemcpy(e->soa.p, soa_host, sizeof(double) * kSoaFields * n, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemset(e->counters.p, 0, sizeof(unsigned long long) * 8) != cudaSuccess)
        rc = SFHK_E_CUDA;
    if (!rc) rc = launch_n0_from_soa((const double*)e->soa.p, n, (int*)e->n0.p, 0);
    if (!rc) rc = ensemble_finish(e, 0);
    if (!rc && cudaStreamSynchronize(0) != cudaSuccess) rc = SFHK_E_CUDA;
    if (rc) {
        ensemble_free(e);
        return rc;
    }
    *out = e;
    return SFHK_OK;
}

int sfhk_ensemble_read(sfhk_ensemble* e, double* soa_host, uint64_t n_traj)
{
    if (!e || !soa_host || (long long)n_traj != e->n) return SFHK_E_INVAL;
    int rc = set_device(e->ctx->device);
    if (rc) return rc;
    SFHK_CUDA_TRY(cudaDeviceSynchronize());
    SFHK_CUDA_TRY(cudaMemcpy(soa_host, e->soa.p, sizeof(double) * kSoaFields * e->n,
                             cudaMemcpyDeviceToHost));
    return SFHK_OK;
}

int sfhk_destroy_ensemble(sfhk_ensemble* e)
{
    if (!e) return SFHK_E_INVAL;
    set_device(e->ctx->device);
    cudaDeviceSynchronize();
    ensemble_free(e);
    return SFHK_OK;
}

int sfhk_propagate(sfhk_ctx* c, sfhk_ensemble* e, const sfhk_run_opts* o, void* stream)
{
    if (!c || !e || e->ctx != c) return SFHK_E_INVAL;
    int rc = check_opts(o);
    if (rc) return rc;
    if ((rc = set_device(c->device))) return rc;
    cudaStream_t s = as_stream(stream);
    if ((rc = prepare_outputs(e, *o, s))) return rc;
    const DevInstance I = make_instance(e, *o);
    SFHK_CUDA_TRY(cudaMemcpyAsync(e->inst.p, &I, sizeof I, cudaMemcpyHostToDevice, s));
    int slots = 0, nc = 0;
    poly_slots(&e, 1, &slots, &nc);
    int bt, var, bps;
    shape(c, *o, fixed_form(&I, 1, o->precision, slots, nc), &bt, &var, &bps);
    SFHK_CUDA_TRY(record_event(e->ev_start, s));
    rc = launch_propagate(o->precision, var, (const DevInstance*)e->inst.p,
                          (const WorkItem*)e->items.p, e->n_items, (unsigned int*)e->qctr.p, bt,
                          bps, c->sm_count, s, slots, nc,
                          fixed_form(&I, 1, o->precision, slots, nc));
    if (rc) return rc;
    e->fixed = fixed_form(&I, 1, o->precision, slots, nc) != kPotAny;
    SFHK_CUDA_TRY(record_event(e->ev_stop, s));
    SFHK_CUDA_TRY(record_event(e->ev_done, s));
    e->have_result = true;
    set_nonfinite_limit(e, *o);
    return SFHK_OK;
}

int sfhk_propagate_batch(sfhk_ctx* c, sfhk_ensemble* const* ens, int n_ens,
                         const sfhk_run_opts* o, void* stream)
{
    if (!c || !ens || n_ens < 1) return SFHK_E_INVAL;
    for (int i = 0; i < n_ens; ++i)
        if (!ens[i] || ens[i]->ctx != c) return SFHK_E_INVAL;
    int rc = check_opts(o);
    if (rc) return rc;
    int slots = 0, nc = 0;
    if ((rc = poly_slots(ens, n_ens, &slots, &nc))) return rc;
    if ((rc = set_device(c->device))) return rc;
    cudaStream_t s = as_stream(stream);
    long long total_items = 0;
    int max_nt = 1;
    for (int i = 0; i < n_ens; ++i) {
        total_items += ens[i]->n_items;
        max_nt = std::max(max_nt, ens[i]->pulse->nt);
    }
    if (total_items > 2147483647ll) return SFHK_E_INVAL;
    // batch scratch: instances, items (x2), keys, perm, hist, nt per instance, counter;
    // stream-ordered, so the call stays asynchronous
    const size_t bytes = sizeof(DevInstance) * n_ens + 2 * sizeof(WorkItem) * total_items +
                         2 * sizeof(int) * total_items + sizeof(int) * (max_nt + 1) +
                         sizeof(int) * n_ens + 4096;
    if (c->budget != 0 && c->used.load() + bytes > c->budget) return SFHK_E_NOMEM;
    void* scratch = nullptr;
    if (cudaMallocAsync(&scratch, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return SFHK_E_NOMEM;
    }
    char* base = (char*)scratch;
    auto take = [&](size_t b) {
        char* r = base;
        base += (b + 255) & ~size_t(255);
        return (void*)r;
    };
    DevInstance* d_inst = (DevInstance*)take(sizeof(DevInstance) * n_ens);
    WorkItem* d_items = (WorkItem*)take(sizeof(WorkItem) * total_items);
    WorkItem* d_sorted = (WorkItem*)take(sizeof(WorkItem) * total_items);
    int* d_keys = (int*)take(sizeof(int) * total_items);
    int* d_perm = (int*)take(sizeof(int) * total_items);
    int* d_hist = (int*)take(sizeof(int) * (max_nt + 1));
    int* d_nt = (int*)take(sizeof(int) * n_ens);
    unsigned int* d_ctr = (unsigned int*)take(sizeof(unsigned int) * 4);
    std::vector<DevInstance> hI(n_ens);
    std::vector<int> hnt(n_ens);
    long long off = 0;
    for (int i = 0; i < n_ens && !rc; ++i) {
        sfhk_ensemble* e = ens[i];
        rc = prepare_outputs(e, *o, s);
        if (rc) break;
        hI[i] = make_instance(e, *o);
        hnt[i] = e->pulse->nt;
        rc = launch_build_items((const int*)e->perm.p, (const int*)e->n0.p, e->n, i,
                                d_items + off, s);
        off += e->n_items;
    }
    // pageable host sources: the copies have read them when the calls return
    if (!rc && (cudaMemcpyAsync(d_inst, hI.data(), sizeof(DevInstance) * n_ens,
                                cudaMemcpyHostToDevice, s) != cudaSuccess ||
                cudaMemcpyAsync(d_nt, hnt.data(), sizeof(int) * n_ens, cudaMemcpyHostToDevice,
                                s) != cudaSuccess))
        rc = SFHK_E_CUDA;
    if (!rc)
        rc = launch_sort_items(d_items, (int)total_items, d_nt, d_sorted, d_keys, d_perm, d_hist,
                               max_nt, s);
    int bt, var, bps;
    shape(c, *o, fixed_form(hI.data(), n_ens, o->precision, slots, nc), &bt, &var, &bps);
    for (int i = 0; i < n_ens && !rc; ++i)
        if (record_event(ens[i]->ev_start, s) != cudaSuccess) rc = SFHK_E_CUDA;
    if (!rc)
        rc = launch_propagate(o->precision, var, d_inst, d_sorted, (int)total_items, d_ctr, bt,
                              bps, c->sm_count, s, slots, nc,
                              fixed_form(hI.data(), n_ens, o->precision, slots, nc));
    const bool fixed = fixed_form(hI.data(), n_ens, o->precision, slots, nc) != kPotAny;
    for (int i = 0; i < n_ens && !rc; ++i) {
        ens[i]->fixed = fixed;
        if (record_event(ens[i]->ev_stop, s) != cudaSuccess ||
            record_event(ens[i]->ev_done, s) != cudaSuccess)
            rc = SFHK_E_CUDA;
        ens[i]->have_result = true;
        set_nonfinite_limit(ens[i], *o);
    }
    cudaFreeAsync(scratch, s);
    return rc;
}

}  // extern "C"

struct sfhk_batch {
    sfhk_ctx* ctx = nullptr;
    std::vector<sfhk_ensemble*> ens;
    sfhk_run_opts opts;
    sfhk::DeviceBuf buf;
    sfhk::DevInstance* d_inst = nullptr;
    sfhk::WorkItem *d_items = nullptr, *d_sorted = nullptr;
    int *d_keys = nullptr, *d_perm = nullptr, *d_hist = nullptr, *d_nt = nullptr;
    unsigned int* d_ctr = nullptr;
    long long total_items = 0;
    int max_nt = 1;
    int poly_slots = 0;
    int poly_nc = 0;                 // common centre count of the polyatomic targets
    int fixed = kPotAny;             // the FixedParams instantiation it runs (fixed_form)
};

extern "C" {

int sfhk_batch_create(sfhk_ctx* c, sfhk_ensemble* const* ens, int n_ens, const sfhk_run_opts* o,
                      sfhk_batch** out)
{
    if (!c || !ens || n_ens < 1 || !out) return SFHK_E_INVAL;
    for (int i = 0; i < n_ens; ++i)
        if (!ens[i] || ens[i]->ctx != c) return SFHK_E_INVAL;
    int rc = check_opts(o);
    if (rc) return rc;
    int slots = 0, nc = 0;
    if ((rc = poly_slots(ens, n_ens, &slots, &nc))) return rc;
    if ((rc = set_device(c->device))) return rc;
    sfhk_batch* b = new (std::nothrow) sfhk_batch;
    if (!b) return SFHK_E_NOMEM;
    b->ctx = c;
    b->poly_slots = slots;
    b->poly_nc = nc;
    b->ens.assign(ens, ens + n_ens);
    b->opts = *o;
    b->opts.dump_final = 0;
    b->opts.record_returns = 0;
    for (int i = 0; i < n_ens; ++i) {
        b->total_items += ens[i]->n_items;
        b->max_nt = std::max(b->max_nt, ens[i]->pulse->nt);
    }
    if (b->total_items > 2147483647ll) {
        delete b;
        return SFHK_E_INVAL;
    }
    const size_t bytes = sizeof(DevInstance) * n_ens + 2 * sizeof(WorkItem) * b->total_items +
                         2 * sizeof(int) * b->total_items + sizeof(int) * (b->max_nt + 1) +
                         sizeof(int) * n_ens + 4096;
    if ((rc = c->alloc(b->buf, bytes))) {
        delete b;
        return rc;
    }
    char* base = (char*)b->buf.p;
    auto take = [&](size_t n) {
        char* r = base;
        base += (n + 255) & ~size_t(255);
        return (void*)r;
    };
    b->d_inst = (DevInstance*)take(sizeof(DevInstance) * n_ens);
    b->d_items = (WorkItem*)take(sizeof(WorkItem) * b->total_items);
    b->d_sorted = (WorkItem*)take(sizeof(WorkItem) * b->total_items);
    b->d_keys = (int*)take(sizeof(int) * b->total_items);
    b->d_perm = (int*)take(sizeof(int) * b->total_items);
    b->d_hist = (int*)take(sizeof(int) * (b->max_nt + 1));
    b->d_nt = (int*)take(sizeof(int) * n_ens);
    b->d_ctr = (unsigned int*)take(sizeof(unsigned int) * 4);
    std::vector<DevInstance> hI(n_ens);
    std::vector<int> hnt(n_ens);
    for (int i = 0; i < n_ens; ++i) {
        hI[i] = make_instance(ens[i], b->opts);
        hnt[i] = ens[i]->pulse->nt;
    }
    b->fixed = fixed_form(hI.data(), n_ens, b->opts.precision, b->poly_slots, b->poly_nc);
    if (cudaMemcpy(b->d_inst, hI.data(), sizeof(DevInstance) * n_ens, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_nt, hnt.data(), sizeof(int) * n_ens, cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        c->release(b->buf);
        delete b;
        return SFHK_E_CUDA;
    }
    *out = b;
    return SFHK_OK;
}

int sfhk_batch_launch(sfhk_batch* b, void* stream)
{
    if (!b) return SFHK_E_INVAL;
    int rc = set_device(b->ctx->device);
    if (rc) return rc;
    cudaStream_t s = as_stream(stream);
    long long off = 0;
    for (size_t i = 0; i < b->ens.size(); ++i) {
        sfhk_ensemble* e = b->ens[i];
        SFHK_CUDA_TRY(cudaMemsetAsync(e->vz.p, 0, sizeof(double) * e->pulse->nt, s));
        SFHK_CUDA_TRY(cudaMemsetAsync(e->counters.p, 0, sizeof(unsigned long long) * 3, s));
        SFHK_CUDA_TRY(cudaMemsetAsync((unsigned long long*)e->counters.p + 4, 0,
                                      sizeof(unsigned long long) * 2, s));
        rc = launch_build_items((const int*)e->perm.p, (const int*)e->n0.p, e->n, (int)i,
                                b->d_items + off, s);
        if (rc) return rc;
        off += e->n_items;
        e->dumped = false;
        e->have_result = true;
        e->fixed = b->fixed != kPotAny;
        set_nonfinite_limit(e, b->opts);
    }
    rc = launch_sort_items(b->d_items, (int)b->total_items, b->d_nt, b->d_sorted, b->d_keys,
                           b->d_perm, b->d_hist, b->max_nt, s);
    if (rc) return rc;
    int bt, var, bps;
    shape(b->ctx, b->opts, b->fixed, &bt, &var, &bps);
    // the kernel is timed with the ensembles' events (also inside a captured graph)
    for (sfhk_ensemble* e : b->ens) SFHK_CUDA_TRY(record_event(e->ev_start, s));
    rc = launch_propagate(b->opts.precision, var, b->d_inst, b->d_sorted, (int)b->total_items,
                          b->d_ctr, bt, bps, b->ctx->sm_count, s, b->poly_slots, b->poly_nc,
                          b->fixed);
    if (rc) return rc;
    for (sfhk_ensemble* e : b->ens) {
        SFHK_CUDA_TRY(record_event(e->ev_stop, s));
        SFHK_CUDA_TRY(record_event(e->ev_done, s));
    }
    return SFHK_OK;
}

int sfhk_batch_destroy(sfhk_batch* b)
{
    if (!b) return SFHK_E_INVAL;
    set_device(b->ctx->device);
    cudaDeviceSynchronize();
    b->ctx->release(b->buf);
    delete b;
    return SFHK_OK;
}

int sfhk_autotune(sfhk_ctx* c, sfhk_ensemble* e, const sfhk_run_opts* o, int max_items,
                  int* choice)
{
    if (!c || !e || e->ctx != c) return SFHK_E_INVAL;
    int rc = check_opts(o);
    if (rc) return rc;
    if ((rc = set_device(c->device))) return rc;
    const int items = (max_items > 0 && max_items < e->n_items) ? max_items : e->n_items;
    sfhk_run_opts oo = *o;
    oo.dump_final = 0;
    oo.record_returns = 0;
    if ((rc = prepare_outputs(e, oo, 0))) return rc;
    const DevInstance I = make_instance(e, oo);
    SFHK_CUDA_TRY(cudaMemcpy(e->inst.p, &I, sizeof I, cudaMemcpyHostToDevice));
    int slots = 0, nc = 0;
    poly_slots(&e, 1, &slots, &nc);
    const int blocks[3] = {32, 64, 128};
    // one timed launch per shape (after a warm-up launch), then the three
    // fastest shapes timed twice more: launch times of close shapes differ by
    // about 1 %, the size of the run-to-run spread
    auto time_shape = [&](int v, int b, float* ms) -> int {
        SFHK_CUDA_TRY(cudaEventRecord(e->ev_start, 0));
        const int r = launch_propagate(o->precision, v, (const DevInstance*)e->inst.p,
                                       (const WorkItem*)e->items.p, items,
                                       (unsigned int*)e->qctr.p, b, 0, c->sm_count, 0, slots,
                                       nc, fixed_form(&I, 1, o->precision, slots, nc));
        if (r) return r;
        SFHK_CUDA_TRY(cudaEventRecord(e->ev_stop, 0));
        SFHK_CUDA_TRY(cudaEventSynchronize(e->ev_stop));
        SFHK_CUDA_TRY(cudaEventElapsedTime(ms, e->ev_start, e->ev_stop));
        return SFHK_OK;
    };
    struct Shape { float ms; int v, b; };
    std::vector<Shape> shapes;
    for (int v = 0; v < kPropVariants; ++v)
        for (int b : blocks) {
            float ms = 0.0f;
            for (int rep = 0; rep < 2; ++rep)        // the first launch warms up
                if ((rc = time_shape(v, b, &ms))) return rc;
            shapes.push_back({ms, v, b});
        }
    std::sort(shapes.begin(), shapes.end(),
              [](const Shape& x, const Shape& y) { return x.ms < y.ms; });
    const size_t top = std::min<size_t>(3, shapes.size());
    for (size_t k = 0; k < top; ++k)
        for (int rep = 0; rep < 2; ++rep) {
            float ms = 0.0f;
            if ((rc = time_shape(shapes[k].v, shapes[k].b, &ms))) return rc;
            shapes[k].ms = std::min(shapes[k].ms, ms);
        }
    std::sort(shapes.begin(), shapes.begin() + top,
              [](const Shape& x, const Shape& y) { return x.ms < y.ms; });
    const int bb = shapes[0].b, bv = shapes[0].v;
    // the shape of the form the ensemble's launches run
    int* t = c->tuned[o->precision][fixed_form(&I, 1, o->precision, slots, nc)];
    t[0] = bb;
    t[1] = bv;
    t[2] = 0;
    e->have_result = false;
    if (choice) {
        choice[0] = bb;
        choice[1] = bv + 1;
        choice[2] = propagate_variant_maxreg(bv);
    }
    return SFHK_OK;
}

int sfhk_dipole(sfhk_ctx* c, sfhk_ensemble* e, double* vz_host, size_t nt, double* t_origin,
                double* dt)
{
    if (!c || !e || !vz_host || nt != (size_t)e->pulse->nt || !e->have_result) return SFHK_E_INVAL;
    int rc = set_device(c->device);
    if (rc) return rc;
    SFHK_CUDA_TRY(cudaEventSynchronize(e->ev_done));
    if (e->check_nonfinite) {
        unsigned long long h[2] = {0, 0};
        SFHK_CUDA_TRY(cudaMemcpy(h, e->counters.p, sizeof h, cudaMemcpyDeviceToHost));
        if (h[1] > e->max_nonfinite) return SFHK_E_NUMERIC;
    }
    SFHK_CUDA_TRY(cudaMemcpy(vz_host, e->vz.p, sizeof(double) * nt, cudaMemcpyDeviceToHost));
    if (t_origin) *t_origin = e->pulse->t_origin;
    if (dt) *dt = e->pulse->dt;
    return SFHK_OK;
}

int sfhk_dipole_device(sfhk_ensemble* e, const double** vz_dev, size_t* nt)
{
    if (!e || !vz_dev) return SFHK_E_INVAL;
    *vz_dev = (const double*)e->vz.p;
    if (nt) *nt = (size_t)e->pulse->nt;
    return SFHK_OK;
}

int sfhk_stats_get(sfhk_ensemble* e, sfhk_stats* out)
{
    if (!e || !out) return SFHK_E_INVAL;
    int rc = set_device(e->ctx->device);
    if (rc) return rc;
    std::memset(out, 0, sizeof *out);
    unsigned long long h[6] = {0, 0, 0, 0, 0, 0};
    if (e->have_result) SFHK_CUDA_TRY(cudaEventSynchronize(e->ev_done));
    SFHK_CUDA_TRY(cudaDeviceSynchronize());
    SFHK_CUDA_TRY(cudaMemcpy(h, e->counters.p, sizeof h, cudaMemcpyDeviceToHost));
    out->n_traj = (uint64_t)e->n;
    out->n_filtered = h[0];
    out->n_nonfinite = h[1];
    out->traj_steps = h[2];
    out->n_invalid = h[3];
    out->n_unstable = h[4];
    out->recomb_evals = h[5];
    out->fixed_params = e->have_result && e->fixed ? 1 : 0;
    out->nt = e->pulse->nt;
    float ms = 0.0f;
    if (e->have_result && cudaEventElapsedTime(&ms, e->ev_start, e->ev_stop) == cudaSuccess)
        out->kernel_ms = ms;
    else
        cudaGetLastError();
    // over the caller's limit: the counters are still returned
    if (e->have_result && e->check_nonfinite && out->n_nonfinite > e->max_nonfinite)
        return SFHK_E_NUMERIC;
    return SFHK_OK;
}

int sfhk_returns(sfhk_ensemble* e, double* host, uint64_t n_traj)
{
    if (!e || !host || (long long)n_traj != e->n || !e->returns_kept || !e->returns.p)
        return SFHK_E_INVAL;
    int rc = set_device(e->ctx->device);
    if (rc) return rc;
    SFHK_CUDA_TRY(cudaEventSynchronize(e->ev_done));
    SFHK_CUDA_TRY(cudaMemcpy(host, e->returns.p, sizeof(double) * 2 * e->n,
                             cudaMemcpyDeviceToHost));
    return SFHK_OK;
}

int sfhk_final_state(sfhk_ensemble* e, double* host, uint64_t n_traj)
{
    if (!e || !host || (long long)n_traj != e->n || !e->dumped || !e->dump.p) return SFHK_E_INVAL;
    int rc = set_device(e->ctx->device);
    if (rc) return rc;
    SFHK_CUDA_TRY(cudaEventSynchronize(e->ev_done));
    SFHK_CUDA_TRY(cudaMemcpy(host, e->dump.p, sizeof(double) * kFinalFields * e->n,
                             cudaMemcpyDeviceToHost));
    return SFHK_OK;
}

int sfhk_spectrum(const double* vz, size_t nt, double dt, double t_origin, double tau_H,
                  double* omega_out, double* yield_out, double* phase_out, size_t n_out,
                  int device_ptrs, void* stream)
{
    if (!vz || nt < 2 || nt > (size_t)(1 << 27) || n_out > nt || n_out == 0 || !(dt > 0.0) ||
        !(tau_H > 0.0))
        return SFHK_E_INVAL;
    cudaStream_t s = as_stream(stream);
    const int N = (int)nt, K = (int)n_out;
    if (device_ptrs) {
        void* tw = nullptr;
        SFHK_CUDA_TRY(cudaMallocAsync(&tw, (sizeof(double2) + sizeof(double)) * N, s));
        int rc = launch_spectrum(vz, N, dt, t_origin, tau_H, omega_out, yield_out, phase_out, K,
                                 (double2*)tw, s);
        cudaFreeAsync(tw, s);
        return rc;
    }
    // layout: twiddle (double2, at the allocation's alignment) | windowed
    // samples | dipole | omega | yield | phase
    void* buf = nullptr;
    const size_t bytes = (sizeof(double2) + sizeof(double)) * N + sizeof(double) * N +
                         3 * sizeof(double) * K;
    SFHK_CUDA_TRY(cudaMallocAsync(&buf, bytes, s));
    double2* tw = (double2*)buf;
    double* dvz = (double*)(tw + N) + N;
    double* om = dvz + N;
    double* yl = om + K;
    double* phs = yl + K;
    int rc = SFHK_OK;
    if (cudaMemcpyAsync(dvz, vz, sizeof(double) * N, cudaMemcpyHostToDevice, s) != cudaSuccess)
        rc = SFHK_E_CUDA;
    if (!rc) rc = launch_spectrum(dvz, N, dt, t_origin, tau_H, om, yl, phs, K, tw, s);
    if (!rc && omega_out &&
        cudaMemcpyAsync(omega_out, om, sizeof(double) * K, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = SFHK_E_CUDA;
    if (!rc && yield_out &&
        cudaMemcpyAsync(yield_out, yl, sizeof(double) * K, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = SFHK_E_CUDA;
    if (!rc && phase_out &&
        cudaMemcpyAsync(phase_out, phs, sizeof(double) * K, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        rc = SFHK_E_CUDA;
    cudaFreeAsync(buf, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) rc = SFHK_E_CUDA;
    return rc;
}

}  // extern "C"
