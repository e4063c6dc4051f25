// op.h -- the device operator (dirac_op) and the launch helpers shared by the C ABI
// implementation (capi.cu) and the CUDA-graph step driver (graph.cu).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "device.h"
#include "internal.h"

namespace dg {

// Krylov workspace in one working precision (prec 0: complex128, 1: complex64): the vectors
// of BiCGSTAB, its scalar state and the operator data it multiplies with.
struct Krylov {
    int prec = 0;
    void *b = nullptr, *x = nullptr, *r = nullptr, *rh = nullptr, *p = nullptr, *v = nullptr, *ph = nullptr,
         *sv = nullptr, *sh = nullptr, *t = nullptr;
    KState* ks = nullptr;
    const void *S = nullptr, *H = nullptr, *W = nullptr, *U = nullptr, *L = nullptr;
    const void *Urow = nullptr, *Dinv = nullptr;   // lane-per-channel preconditioner data
};

struct GraphDriver;   // graph.cu

// Buffers of one double-float assembly (precision 2): evaluation time, pulse factors, combined
// bands and the coupling values they produce.  Set 0 is the operator's own; set 1 exists when the
// next step's assembly overlaps the current step's solve.
struct AsmSet {
    double* t_eval = nullptr;
    double* s = nullptr;
    float2 *Gdf = nullptr, *Kdf = nullptr, *KTdf = nullptr;
    float *Wh = nullptr, *Wl = nullptr;
    float* Ghi = nullptr;   // hi words of Gdf as plain floats (factorised apply, subgroup form)
};

}  // namespace dg

namespace dg { struct SpecState; }

struct dirac_op {
    dg::Basis B;                 // host copy of the basis data the operator needs
    dirac_pulse pulse{};
    dirac_solver_opts opts{};
    cudaStream_t st = nullptr;
    int device = 0;
    int64_t n = 0, npairs = 0;
    // block partials written by each kind of launch (the reductions must read exactly these):
    // nparts_apply: 128-row tiles (FP64 apply, observables); nparts_own: the owner/gather passes
    int nparts_apply = 0, nparts_own = 0, nparts_vec = 0, nparts_prec = 0, nparts_prec32 = 0;
    int prec_warps = 0;          // same-kappa channel groups (lane-per-channel preconditioner)
    // preconditioner schedules, picked by timing at setup: 0 one lane per channel (complex64 only),
    // 1 one warp per channel, 2 one warp per channel with shared-memory staging
    int prec_sched32 = 0, prec_sched64 = 1;
    bool prec_sm_ok = false;     // the staged kernel fits this radial size
    bool prec_rot_ok = false;    // the rotated-lane kernel is set up (band width 13)
    float prec_ms32[4] = {0, 0, 0, 0}, prec_ms64[4] = {0, 0, 0, 0};
    int config_gen = 0;          // bumped when a launch choice changes (captured graphs are rebuilt)
    int *wks = nullptr, *wfirst = nullptr, *wcnt = nullptr;
    std::vector<void*> allocs;
    size_t bytes = 0;
    dg::OpView ov{};
    dg::PulseView pv{};
    double* G = nullptr;         // G^n_l(t) bands
    double* s = nullptr;         // time factors
    double* t_eval = nullptr;
    double* K = nullptr;         // combined radial bands K_l(k', k)(t)
    double* W = nullptr;         // coupling values, FP64 (precision 0 and 1)
    // precision 2: double-float operator data (hi/lo float pairs)
    float2 *Gdf = nullptr, *Kdf = nullptr, *KTdf = nullptr, *Sdf = nullptr, *Htdf = nullptr;
    float2 *SdfT = nullptr, *HdfT = nullptr;   // S, tau H0 rows innermost (order 7), for the gather pass
    float *S32T = nullptr, *H32T = nullptr;     // S, H0 in FP32 rows innermost, for the complex64 owner pass
    float *Wh = nullptr, *Wl = nullptr;   // coupling hi words (also the FP32 values) and lo words
    float4* cab_df = nullptr;
    // factorised complex64 apply of the inner solve (dirac_op_set_factorised)
    int fact32 = 0;              // 0 stored coupling, 1 subgroup form, 2 per-channel form
    dg::RadChunk* rad_chunks = nullptr;
    int nrad = 0;
    dg::RadPack* rad_lanes = nullptr;    // subgroup form: pairs of kappa chunks sharing FLANE lanes
    int nrad_lanes = 0;
    dg::FactSub* fsub = nullptr;         // subgroup form: FSG outputs of one mu and their items
    int nfsub = 0, fsub_max = 1;         // subgroups, the largest item count
    int* fitem_off = nullptr;            // item -> partner * L + multipole
    float4* fitem_coef = nullptr;        // item -> FSG coefficient sets (U, V, U', V')
    float2* Zf = nullptr;        // band products of one radial tile
    float* Ghi = nullptr;        // the current buffer set's G hi words (subgroup form)
    // grouped double-float assembly (null when a group has more than ASM_MAX_NL multipoles)
    dg::AsmChunk* asm_chunks = nullptr;
    int asm_nchunks = 0;
    int* asm_gpair = nullptr;
    float4* asm_gcoef = nullptr;
    float4* xsplit = nullptr;    // split input vector; u = psi + x in the fused residual
    float4* vsplit = nullptr;    // v = psi - x in the fused residual
    float* W32 = nullptr;        // their FP32 rounding (mixed precision only)
    dg::Krylov k64, k32;         // FP64 solve (outer loop in mixed precision), FP32 inner solve
    double2* part_d = nullptr;
    double* part_n = nullptr;
    double* part_n2 = nullptr;
    float4* part_own = nullptr;  // transposed partial products of the complex64 owner/gather apply
    float4* part_rdf = nullptr;  // ... of the double-float refinement residual (2 per row)
    float4* part_bdf = nullptr;  // ... of b = A_- psi on a step's first refinement pass
    float2* psi32 = nullptr;     // psi in FP32 and b = A_- psi (tolerance scale) of the residual pass
    float2* b32 = nullptr;
    // offsets of the residual owner pass's accumulators: static envelopes of the pulse matrices
    // ([L][4][n1], row/column maxima and their 13-row window maxima), u-window sums, offset bytes
    float* own_E = nullptr;
    float* own_Ew = nullptr;
    float* own_US = nullptr;
    unsigned char* own_sig = nullptr;
    int* need_b = nullptr;       // device flag: the next residual pass also forms ||b||^2
    int* ch_two_mu = nullptr;    // [nch] 2 mu of each channel (learned-guess features)
    dirac_guess* net = nullptr;  // learned initial guess (guess option 2), not owned
    float *gx = nullptr, *gs = nullptr, *gout = nullptr;   // its features, scales and outputs
    float* gfield = nullptr;     // its six field factors (device) and, in a graph, the gate flag
    int* ggate = nullptr;
    int* dev_err = nullptr;      // set by kernels whose bounded waits ran out
    unsigned int* bounds_err = nullptr;   // bit per check site, set by debug (DG_BOUNDS) builds only
    double2* part_d2 = nullptr;
    double2* psi0_g = nullptr;   // ground state of the kappa=-1 mu=+1/2 channel (2 n1)
    double* bvec = nullptr;      // bound eigenvectors per kappa slot, [vector][2 n1] (built on first use)
    int* bstart = nullptr;       // first vector of each kappa slot (2 kappa_max + 1)
    double* part_pb = nullptr;   // per-channel bound populations
    int nbound = 0;
    int ground_ch = -1;
    // kernel-phase timers (CUDA events on the op's stream) and the launch counter
    bool profiling = false;
    int64_t launches = 0;
    double phase_ms[DIRAC_NPHASE] = {0};
    int64_t phase_n[DIRAC_NPHASE] = {0};
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> pending;
    std::vector<cudaEvent_t> event_pool;
    dg::GraphDriver* graph = nullptr;   // captured multi-step driver (dirac_run), built on first use
    // overlapped assembly (dirac_op_set_overlap): the next step's coupling values are assembled on
    // st_asm into the other buffer set while the current step solves
    bool overlap = false;
    int resid_mode = 0;                  // dirac_op_set_residual_mode (0 automatic, 1 Dot2, 2 offsets)
    dg::AsmSet aset[2];
    int acur = 0;                        // the set op->Wh / op->Wl currently point to
    cudaStream_t st_asm = nullptr;
    cudaEvent_t ev_asm[2] = {nullptr, nullptr}, ev_use[2] = {nullptr, nullptr};
    cudaEvent_t ev_res = nullptr;        // the current step's first residual pass, done
    dg::SpecState* spec = nullptr;       // photoelectron spectrum: eigenpairs of one window (first use)
};

namespace dg {

int grid_for(int64_t n, int bs);
void collect_phases(dirac_op* op);
dirac_status check_launch(const char* what);
int apply_parts(const dirac_op* op, const Krylov& K);   // partials of k_apply_launch on K
int prec_parts(const dirac_op* op, const Krylov& K);    // partials of k_precond_launch on K
void k_apply_launch(dirac_op* op, const Krylov& K, int sign, const void* x, void* y, const void* bsub,
                    const void* dv, double2* pdot, double* pnrm, const KState* skip);
void launch_assemble(dirac_op* op);
void launch_assemble_set(dirac_op* op, cudaStream_t st, const AsmSet& a);
void apply_accurate(dirac_op* op, int sign, const void* x, void* y, const void* bsub, double* pnrm);
void rhs_accurate(dirac_op* op, const void* psi);
void residual_accurate(dirac_op* op, const void* psi);
void k_precond_launch(dirac_op* op, const Krylov& K, int mode, const KState* ks, const void* r, const void* v,
                      void* io, void* z, double* pn);
void finish(dirac_op* op, KState* ks, int what, int np, const double2* pd, const double* pn, int max_iter);
void vcopy(dirac_op* op, const Krylov& K, const void* a, void* b);
void vzero(dirac_op* op, const Krylov& K, void* a);
dirac_status read_state(dirac_op* op, const Krylov& K, KState& hs);
dirac_status check_dev_err(dirac_op* op, const char* what);
dirac_status bicgstab_iteration(dirac_op* op, const Krylov& K, int max_iter, bool mid_check);
void bicgstab_begin(dirac_op* op, const Krylov& K, int max_iter, bool rel_start = false);
void set_error(const std::string& msg);
void graph_free(dirac_op* op);
dirac_status bound_population(dirac_op* op, const double2* psi, double* out);
dirac_status eig_window(dirac_op* op, double vl, double vu, std::vector<double>& hvec, std::vector<double>& hE,
                        std::vector<int>& hstart);
void spec_free(dirac_op* op);
dirac_status obs_scratch_address(int device, double2** out);   // static scratch of dirac_observables_static
dirac_status guess_buffers(dirac_op* op);
dirac_status guess_into(dirac_op* op, const double2* p0, const double2* h1, const double2* h2, const double2* h3,
                        double t_start, int step, double2* x, const int* gate, cudaStream_t st,
                        const float* field);

}  // namespace dg
