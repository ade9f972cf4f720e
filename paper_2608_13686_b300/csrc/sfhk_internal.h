// sfhk_internal.h -- library-internal types shared by the host runtime and
// the kernels of libsfhk (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <cstdio>
#include <mutex>
#include <vector>

#include "../../include/sfhk.h"

namespace sfhk {

// The form of the two-centre potential an integrator is compiled for:
// kPotAny decides the kind (molecular or the harmonic test potential) and
// the screening per instance at run time; kPotMolecule is the molecular
// potential with the screening decided per instance; kPotBare and
// kPotScreened fix the screening for the whole launch as well.
constexpr int kPotAny = 0, kPotBare = 1, kPotScreened = 2, kPotMolecule = 3;

constexpr int kWarp = 32;
constexpr int kFinalFields = 47;   // see sfhk_final_state
constexpr int kSoaFields = 12;     // see sfhk_load_ensemble

// ------------------------------------------------------------------ device views
// Target constants as the kernels use them.  Recombination constants per
// primitive k (coherent-state width gamma, b = gamma/2, c = a_k + b):
//   <phi_k(.-A)| k_z |p,q> = K4 (p_z - i gamma d_z) exp(K1 |d|^2 + K2 |p|^2 + i K3 p.d),
//   d = q - A, K1 = -a b / c, K2 = -1/(4c), K3 = -a/c,
//   K4 = N coef_k (gamma/pi)^{3/4} (pi/c)^{3/2} a/c.
struct DevTarget {
    int kind;
    int n_prim;
    int screened;          // Z0 != Z_inf
    double half_R, Zinf, dZ, alpha, a2, Ip, w2;
    double norm;           // orbital normalisation N
    double pexp[SFHK_MAX_PRIM], pcoef[SFHK_MAX_PRIM];
    int pkind[SFHK_MAX_PRIM];   // SFHK_PRIM_S / _P_SIGMA / _P_PI / _P_DIR
    double pi_azimuth;          // chi of the pi lobe about the axis
    // polyatomic targets (kind SFHK_POT_POLYATOMIC)
    int n_centres;
    int n_slots;                // per-lane table rows: centres, then p directions
    double cpos[SFHK_MAX_CENTRES][3];                 // molecular frame
    double cZinf[SFHK_MAX_CENTRES], cdZ[SFHK_MAX_CENTRES], calpha[SFHK_MAX_CENTRES];
    float4 cq_f[SFHK_MAX_CENTRES];                    // (Z_inf, dZ, alpha, 0) in FP32
    // centres 2k and 2k+1 side by side: (Zinf, Zinf', dZ, dZ'), (alpha, alpha', 0, 0)
    float4 cq2_f[SFHK_MAX_CENTRES / 2][2];
    int pcentre[SFHK_MAX_PRIM];
    double pdir[SFHK_MAX_PRIM][3];                    // unit, molecular frame
};

struct DevRecomb {
    double K1[SFHK_MAX_PRIM], K2[SFHK_MAX_PRIM], K3[SFHK_MAX_PRIM], K4[SFHK_MAX_PRIM];
    float K1f[SFHK_MAX_PRIM], K2f[SFHK_MAX_PRIM], K3f[SFHK_MAX_PRIM], K4f[SFHK_MAX_PRIM];
    // p-type primitives only
    int has_p;
    int kind[SFHK_MAX_PRIM];    // 0 s, 1 sigma p, 2 pi p
    double cchi, schi;          // cos, sin of the pi lobe's azimuth
    double P1[SFHK_MAX_PRIM], P2[SFHK_MAX_PRIM], P3[SFHK_MAX_PRIM];
    float P1f[SFHK_MAX_PRIM], P2f[SFHK_MAX_PRIM], P3f[SFHK_MAX_PRIM];
};

// One ensemble as seen by the propagation kernel.
struct DevInstance {
    DevTarget tgt;
    DevRecomb rec;
    const double* Eh;      // E at half steps, 2 Nt - 1 entries (FP64)
    const float* Ehf;      // same, FP32
    const double2* ph;     // exp(-i Ip t_n), Nt entries
    const float2* phf;
    const double* soa;     // 12 x n field-major
    const int* perm;       // sorted position -> trajectory index
    const int* n0;         // per trajectory grid index of t0
    double* vz;            // Nt dipole accumulator
    double* dump;          // 47 x n or null
    double* returns;       // 2 x n first returns (step, energy) or null
    double ret_out, ret_in;
    unsigned long long* counters;   // [filtered, nonfinite, steps, invalid, unstable,
                                    //  recombination evaluations]
    long long n;
    int nt;
    double dt, t_origin;
    double scale;          // -2 / N
    double gamma, inv_gamma;
    double cutoff2;        // cutoff^2 on |det| (0 = off), |C|^2 = |det|
    double stab_cut;       // cutoff on max |M_ij| (0 = off)
    double stab_hi;        // tapered filter: stop at this running max (0 = hard cut)
    double inv_log_taper;  // 1 / ln(stab_hi / stab_cut)
    unsigned int* done_items;   // server: work items of this instance finished (or null)
    const int* cancel;          // server: nonzero = skip the remaining items (or null)
};

struct WorkItem {
    int inst;              // index into the instance array
    int first;             // first sorted position
    int count;             // 1..32
    int n_start;           // grid index of the earliest birth in the item
};

// ------------------------------------------------------------------ host objects
struct Ctx;

struct DeviceBuf {
    void* p = nullptr;
    size_t bytes = 0;
};

struct Ctx {
    int device = 0;
    int sm_count = 0;
    size_t budget = 0;
    std::atomic<size_t> used{0};
    std::mutex mu;
    // tuned launch shape per precision and form of the launch's integrator
    // (kPotAny: the generic one; else the fixed-parameter one of that
    // potential form, whose register needs differ): [block_threads, variant,
    // blocks_per_sm] (variant: index into 0 = no cap, 168, 152, ... registers;
    // blocks per SM 0 = as many as fit).  Before tuning: 128 threads, FP64 at
    // the 152-register cap, mixed precision at 168 (the fixed-parameter kernels
    // spill at most 20 B there, up to 112 B at 152)
    int tuned[2][4][3] = {{{128, 2, 0}, {128, 2, 0}, {128, 2, 0}, {128, 2, 0}},
                          {{128, 1, 0}, {128, 1, 0}, {128, 1, 0}, {128, 1, 0}}};
    int alloc(DeviceBuf& b, size_t bytes);
    void release(DeviceBuf& b);
};

struct Target {
    Ctx* ctx;
    sfhk_target_desc desc;
    DevTarget dev;
};

struct Pulse {
    Ctx* ctx;
    sfhk_pulse_desc desc;
    double omega, E0, Tp, t_origin, dt;
    int nt;
    DeviceBuf Eh, Ehf;     // 2 nt - 1 entries
};

struct Ensemble {
    Ctx* ctx;
    const Target* tgt;
    const Pulse* pulse;
    long long n = 0;
    double n_norm = 0;
    DeviceBuf soa, n0, perm, items, ph, phf, vz, dump, counters, returns, pilot;
    int n_items = 0;
    unsigned long long n_invalid = 0;
    bool dumped = false;
    bool returns_kept = false;
    bool have_result = false;
    bool fixed = false;          // the last launch ran the FixedParams integrator
    bool sampled = false;          // created by the device sampler
    bool check_nonfinite = false;  // limit of the last propagation's non-finite count
    unsigned long long max_nonfinite = 0;
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr, ev_done = nullptr;
};

// ------------------------------------------------------------------ launchers
// every launcher adds the number of kernels it enqueued
extern std::atomic<unsigned long long> g_launches;
inline void count_launch(int k = 1) { g_launches.fetch_add((unsigned long long)k); }

// sample / sort (sfhk_sample.cu)
int launch_field_table(const Pulse& P, double* Eh, float* Ehf, cudaStream_t s);
int launch_phase_table(const Pulse& P, double Ip, double2* ph, float2* phf, cudaStream_t s);
int launch_adk_cdf(const Pulse& P, double Ip, double* cdf, cudaStream_t s);
// The same launch writes, after the nt CDF values, the part of a proposal
// draw that depends only on its birth step m (Sec. II.B): row m, at
// cdf + birth_tab_offset(nt) + kBirthTab * m, holds E(t_m), the transverse
// width sigma_m = sqrt(|E|/(2 sqrt(2 Ip))), 1/(2 sigma_m^2), the birth-time
// density W_m / (pi dt sum_n W_n), and sin, cos of k_q t_m + cep for the
// pulse's three terms.  Rows start on a 16-byte boundary.
constexpr int kBirthTab = 10;
__host__ __device__ inline size_t birth_tab_offset(int nt) { return (size_t)((nt + 1) & ~1); }
inline size_t cdf_doubles(int nt) { return birth_tab_offset(nt) + (size_t)kBirthTab * nt; }
// alignment descriptor within its documented ranges
bool align_valid(const sfhk_align_desc& al);
// pilot: sample_pilot_doubles() doubles of scratch, used when the target
// samples ~ |a| (null otherwise)
int launch_sample(const Target& T, const Pulse& P, const sfhk_align_desc& al, long long n,
                  uint64_t seed, uint32_t instance, const double* cdf, double* soa, int* n0,
                  unsigned long long* n_invalid, double* pilot, cudaStream_t s);
size_t sample_pilot_doubles();
int launch_n0_from_soa(const double* soa, long long n, int* n0, cudaStream_t s);
// counting sort of keys in [0, K): writes perm (sorted position -> index)
int launch_counting_sort(const int* keys, long long n, int K, int* perm, int* scratch_hist,
                         cudaStream_t s);
int launch_build_items(const int* perm, const int* n0, long long n, int inst, WorkItem* items,
                       cudaStream_t s);
int launch_sort_items(const WorkItem* in, int n_items, const int* inst_nt, WorkItem* out,
                      int* scratch_keys, int* scratch_perm, int* scratch_hist, int K,
                      cudaStream_t s);
// propagate (sfhk_propagate.cu)
constexpr int kPropVariants = 6;   // register-cap variants of the integrator
// once per device, at context creation: kernel attributes (shared memory)
int configure_kernels();
// The method's prescribed RK4 step and Herman-Kluk width (dt = 0.05,
// gamma = 0.5) with the workloads' filters (prefactor |C| <= 1e4, stability
// taper from max|M| = 1e3 to 2e3).  A mixed-precision launch of diatomic or
// three-centre targets whose every instance has exactly these values runs an
// instantiation of the integrator compiled with them as constants (the same
// arithmetic; the constants then take no registers); any other launch runs
// the generic one.
struct FixedParams {
    static constexpr double dt = 0.05, gamma = 0.5, cutoff = 1e4, stab = 1e3, taper = 2.0;
};
// host: I has exactly FixedParams' values, a molecular target and no
// first-return record (the fixed-parameter integrators keep no such record)
bool fixed_params(const DevInstance& I);
// the FixedParams instantiation a launch runs, as the form of its potential
// (kPotAny: the generic integrator): every instance has the values, mixed
// precision, diatomic targets (their screening: all bare, all screened, or
// decided per instance) or three-centre ones (any form other than kPotAny)
inline int fixed_form(const DevInstance* inst, int n, int precision, int poly_slots, int poly_nc)
{
    if (precision != SFHK_MIXED || n < 1 || (poly_slots > 0 && poly_nc != 3)) return kPotAny;
    int n_screened = 0;
    for (int i = 0; i < n; ++i) {
        if (!fixed_params(inst[i])) return kPotAny;
        n_screened += inst[i].tgt.screened != 0;
    }
    if (poly_slots > 0) return kPotMolecule;
    return n_screened == 0 ? kPotBare : n_screened == n ? kPotScreened : kPotMolecule;
}
// poly_slots > 0: polyatomic instances, launched on the polyatomic kernel
// with that many table rows per lane (the largest n_slots of the instances);
// fixed: the FixedParams instantiation the launch runs (fixed_form)
int launch_propagate(int precision, int variant_index, const DevInstance* insts,
                     const WorkItem* items, int n_items, unsigned int* item_counter,
                     int block_threads, int blocks_per_sm, int sm_count, cudaStream_t s,
                     int poly_slots = 0, int poly_nc = 0, int fixed = kPotAny);
int propagate_occupancy(int precision, int variant_index, int block_threads, int* blocks_per_sm,
                        int fixed = kPotAny);
int propagate_variant_maxreg(int variant_index);   // 0 = no cap
// Server slices stop within one 32-step chunk of their deadline: a warp
// whose time is up at a chunk boundary, with chunks left, parks its item (the
// next chunk's first step and kParkWords values of each lane's state, in the
// precision's type) and the next slice resumes it before taking new items.
constexpr int kParkWords = 58;
struct ParkHdr {
    WorkItem W;
    int nb;                        // first step of the next chunk
    int pad[3];
};
struct ParkBufs {
    const ParkHdr* in_hdr;         // the previous slice's parked items
    const void* in_state;          // [n_in][kParkWords][32]
    int n_in;
    unsigned int* in_ctr;          // zero before the launch
    ParkHdr* out_hdr;              // this slice's parked items
    void* out_state;               // [cap][kParkWords][32]
    unsigned int* out_ctr;         // zero before the launch; ends >= the number parked
    unsigned long long* out_work;  // zero before the launch: the parked items' remaining
                                   // work, Nt x the remaining fraction of each item's steps
                                   // (the units in which the server counts queued items)
    int cap;                       // entries of each buffer; an item beyond it is not parked
};
// warps a slice launch can have at once (the park buffers' capacity): the
// largest over the slice kernels a ring can run
int slice_max_warps(int precision, int variant_index, int block_threads, int sm_count);
// server slice: items ring[(base + i) & mask], i < n_items; warps stop pulling
// new items slice_ns after the first warp started (0 = no limit); *t0 must be
// zero before the launch; *counter ends >= the number of items taken.
// poly_slots > 0: the ring holds polyatomic requests' items, whose centre
// tables have that many rows per lane; fixed (diatomic, mixed precision):
// every request in the ring has FixedParams' values
int launch_propagate_slice(int precision, int variant_index, const DevInstance* insts,
                           const WorkItem* ring, unsigned int mask, unsigned int base,
                           int n_items, unsigned int* counter, unsigned long long slice_ns,
                           unsigned long long* t0, int block_threads, int sm_count,
                           cudaStream_t s, const ParkBufs& park, int poly_slots = 0,
                           bool fixed = false);

// spectrum (sfhk_spectrum.cu)
// Gabor map (sfhk_gabor.cu)
int launch_gabor(const double* vz, int nt, double dt, double t_origin, double sigma,
                 double t_first, double t_step, int n_t, double w_first, double w_step, int n_w,
                 double* out, cudaStream_t s);
int launch_spectrum(const double* vz, int nt, double dt, double t_origin, double tau_H,
                    double* omega, double* yield, double* phase, int n_out, double2* twiddle,
                    cudaStream_t s);

}  // namespace sfhk

// the opaque C handles
struct sfhk_ctx : public sfhk::Ctx {};
struct sfhk_target : public sfhk::Target {};
struct sfhk_pulse : public sfhk::Pulse {};
struct sfhk_ensemble : public sfhk::Ensemble {
    sfhk::DeviceBuf cdf, hist, inst, qctr;
};

namespace sfhk {
// helpers of sfhk_api.cu shared with the server
DevInstance make_instance(sfhk_ensemble* e, const sfhk_run_opts& o);
int prepare_outputs(sfhk_ensemble* e, const sfhk_run_opts& o, cudaStream_t s);
}  // namespace sfhk

// On failure: report, clear the runtime's last-error state (so a later,
// unrelated launch check does not see it again) and return SFHK_E_CUDA.
#define SFHK_CUDA_TRY(expr)                                                         \
    do {                                                                            \
        cudaError_t _e = (expr);                                                    \
        if (_e != cudaSuccess) {                                                    \
            std::fprintf(stderr, "sfhk: %s failed: %s (%s:%d)\n", #expr,            \
                         cudaGetErrorString(_e), __FILE__, __LINE__);               \
            cudaGetLastError();                                                     \
            return SFHK_E_CUDA;                                                     \
        }                                                                           \
    } while (0)

namespace sfhk {
// Record an event on s; inside a stream capture as an external event node, so
// that replays of the captured graph record it too.
inline cudaError_t record_event(cudaEvent_t ev, cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return cudaGetLastError();
    return cs == cudaStreamCaptureStatusActive
               ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal)
               : cudaEventRecord(ev, s);
}
}  // namespace sfhk
