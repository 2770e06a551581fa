/*
 * tevo.h -- C ABI of the GB300 (sm_103a) library for the higher-order
 * time-evolution MPO method of Van Damme, Haegeman, McCulloch and
 * Vanderstraeten, "Efficient higher-order matrix product operators for time
 * evolution", arXiv:2302.14181.
 *
 * The library applies the order-N time-evolution MPO W^(N)(tau) of the paper
 * to a finite matrix product state and fits the product back into an MPS of
 * fixed bond dimension by variational sweeps, one time step after another.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Complex numbers cross the ABI as interleaved pairs of doubles (re, im).
 *    A "complex array of n entries" is a pointer to 2n doubles.
 *  - Host arrays are owned by the caller and only read (or written) during the
 *    call; the library keeps no pointer to them.
 *  - Device memory is owned by the handles (tevo_mpo, tevo_mps) and released by
 *    their destroy calls. It comes from the allocator registered with
 *    tevo_ctx_set_allocator, else from cudaMallocAsync on the context stream.
 *  - Every call is ordered on the context's CUDA stream. Calls that write host
 *    outputs synchronise that stream before returning.
 *  - Every entry point returns 0 on success or a negative TEVO_E* code; no
 *    exception crosses the ABI. tevo_strerror() names a code. After an error the
 *    handles stay valid but the state they hold is unspecified.
 *  - A handle is used by one host thread at a time.
 */
#ifndef TEVO_H
#define TEVO_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* error codes */
#define TEVO_OK 0
#define TEVO_EINVAL (-1)         /* NULL handle/pointer or argument out of range */
#define TEVO_ESHAPE (-2)         /* dimensions of the operands do not fit together */
#define TEVO_ETAU (-3)           /* tau passed to evolve_step differs from the MPO's tau */
#define TEVO_ENOMEM (-4)         /* device or host allocation failed */
#define TEVO_ECUDA (-5)          /* a CUDA runtime call or kernel launch failed */
#define TEVO_ENONFINITE (-6)     /* a NaN or Inf appeared (norm of the fitted state) */
#define TEVO_ETIMEOUT (-7)       /* a bounded device-side wait gave up */
#define TEVO_EUNSUPPORTED (-8)   /* precision/shape combination not built */

/* precision of the environment and apply contractions in evolve_step */
#define TEVO_FP64 0      /* all contractions in fp64 (the plain form) */
#define TEVO_TF32 1      /* tcgen05 kind::tf32, fp32 accumulate; fp64 QR and final sweep */
#define TEVO_TF32X3 2    /* three-pass split tf32 (hi*hi + hi*lo + lo*hi); fp64 QR and final sweep */
#define TEVO_BF16X3 3    /* three-pass split bf16 (hi*hi + hi*lo + lo*hi); fp64 QR and final sweep */
/* OR-ed into a low-precision form: every sweep (and the centre) on the tensor
 * cores, no fp64 rebuild or fp64 sweep; the QR, the norm and the reductions stay
 * fp64. Not the paper's recipe: an extra form for accuracy/speed studies. */
#define TEVO_TC_ONLY 0x100
/* OR-ed into any form: the fp64 contractions (the final sweep and the rebuild
 * of the right environments of the low-precision forms; every sweep of
 * TEVO_FP64) are computed on the bf16 tensor cores by the Ozaki splitting
 * scheme: each operand row is scaled by a power of two and cut into integer
 * digit slices of 7 bits, digit products are exact and their sums are exact in
 * the fp32 accumulator, and the pass results are summed per entry exactly in
 * two 64-bit fixed-point accumulators (integer instructions; 128 bits of
 * range together) and rounded once to fp64.
 * With G slices the dropped part is about (G + 2) 2^(-7 G) of
 * max|row of A| max|row of B| K per entry (G = 8: 56 bits; a native fp64 GEMM
 * has about K 2^-53 of sum |A||B|). Inputs, outputs, the QR, the norm and the
 * reductions stay fp64. TEVO_OZAKI_SLICES(G) picks G in 1..8 (default 8: 56 bits).
 * Not in the paper: a GB300-specific way to run the fp64 sweep, whose fp64
 * pipe is about 1/1600 of its bf16 tensor rate. */
#define TEVO_OZAKI 0x200
#define TEVO_OZAKI_SLICES(g) (TEVO_OZAKI | ((g) << 12))
/* OR-ed into TEVO_FP64 (with or without TEVO_OZAKI): the two-site form of the
 * variational fit (Sec. 2.2, the (i)DMRG row of Table 1 in its two-site form).
 * Each update contracts the target W|psi> on the environments of two
 * neighbouring sites into Theta ((D_l d) x (d D_r)), orthogonalises the columns
 * of Theta by one-sided Jacobi rotations in fp64 (its left singular vectors
 * times the singular values), keeps the D_i of largest norm and re-gauges them
 * with the fp64 Householder QR; the site keeps Q, the environment grows through
 * conj(Q). The bond basis is thus chosen from the target's singular vectors on
 * the pair, so a rank-deficient start needs no completion rule. The Jacobi
 * rounds (N - 1 grid barriers per sweep of rotations, several sweeps per pair)
 * dominate: XXZ L = 32, D = 64, order 3, two sweeps per step take 1.86 s per
 * step against 0.15 s for the single-site fit. Other forms with
 * this flag, and the batched form, are refused (TEVO_EINVAL /
 * TEVO_EUNSUPPORTED). */
#define TEVO_TWO_SITE 0x400

/* variants of the MPO construction (Secs. 3-6 of the paper) */
#define TEVO_MPO_PLAIN 0     /* Algorithm 1 only (Eq. W1 at N = 1, Eq. W2 at N = 2) */
#define TEVO_MPO_EXACT 1     /* Algorithms 1 + 2 */
#define TEVO_MPO_EXTENDED 2  /* Algorithms 3 + 1 + 2 */
#define TEVO_MPO_FULL 3      /* Algorithms 3 + 1 + 2 + 4: the order-N MPO of the Sec. 8.3 table */

typedef struct tevo_ctx_s* tevo_ctx;
typedef struct tevo_mpo_s* tevo_mpo;
typedef struct tevo_mps_s* tevo_mps;

typedef void* (*tevo_alloc_fn)(size_t bytes, void* user);
typedef void (*tevo_free_fn)(void* ptr, void* user);

/* Create a context bound to a CUDA stream (cudaStream_t passed as void*; NULL is
 * the legacy default stream) on the current device. */
int tevo_ctx_create(void* cuda_stream, tevo_ctx* out);
int tevo_ctx_destroy(tevo_ctx ctx);
/* Route device allocations of handles created afterwards through alloc/free
 * (e.g. a framework's caching allocator). alloc must return memory usable on the
 * context stream, aligned to 256 bytes, or NULL on failure. */
int tevo_ctx_set_allocator(tevo_ctx ctx, tevo_alloc_fn alloc, tevo_free_fn free_fn, void* user);
/* Change the stream of an existing context. */
int tevo_ctx_set_stream(tevo_ctx ctx, void* cuda_stream);

/*
 * mpo_build -- W^(N)(tau) for a finite chain (Secs. 2.3-6, Algorithms 1-4,
 * boundary vectors of Eq. boundary), built on the host and uploaded once.
 *
 * The Hamiltonian is given per site in the upper-triangular block form of Eq.
 * jordan_mpo, H = sum_i (D_i + C_i B_{i+1} + C_i A_{i+1} B_{i+2} + ...):
 *   A  : complex [L][chi][chi][d][d]  (left virtual, right virtual, out, in)
 *   B  : complex [L][chi][d][d]       (left virtual, out, in)
 *   C  : complex [L][chi][d][d]       (right virtual, out, in)
 *   Dh : complex [L][d][d]
 * Host pointers, row-major, read during the call only.
 * N in 1..6 is the order, (tau_re, tau_im) the complex step of exp(tau H)
 * (real time t uses tau = -i dt), variant one of TEVO_MPO_*.
 * The site tensors are W_i[w_l][s][s'][w_r] with the level (1,...,1) at index 0;
 * the first site keeps only that row and the last site only that column.
 * Errors: TEVO_EINVAL (bad pointer, L < 2, d < 1, chi < 1, N out of range),
 * TEVO_ENOMEM, TEVO_ECUDA.
 */
int mpo_build(tevo_ctx ctx, int L, int d, int chi, const double* A, const double* B,
              const double* C, const double* Dh, int N, double tau_re, double tau_im,
              int variant, tevo_mpo* out);
/*
 * mpo_build_host -- the same construction as mpo_build, on the host only (no
 * device memory, no CUDA call). Writes the bond dimensions w_0..w_L into w_out
 * (L+1 ints) and, when W_out is not NULL, the site tensors W_i[w_l][d][d][w_r]
 * back to back as complex entries into W_out, which must hold *count entries;
 * *count always receives the total number of complex entries.
 * Errors: TEVO_EINVAL, TEVO_ENOMEM.
 */
int mpo_build_host(int L, int d, int chi, const double* A, const double* B, const double* C,
                   const double* Dh, int N, double tau_re, double tau_im, int variant, int* w_out,
                   double* W_out, size_t* count);

/* bond dimensions w_0..w_L of the built MPO (host array of L+1 ints) */
int mpo_bond_dims(tevo_mpo W, int* w_out);
/* copy site i's tensor W_i[w_l][d][d][w_r] to host (complex, w_l*d*d*w_r entries) */
int mpo_get_site(tevo_mpo W, int i, double* host_out);
int mpo_destroy(tevo_mpo W);

/*
 * mps_init -- product state |v_1> (x) ... (x) |v_L> held at the bond dimensions
 * D_i = min(D, d^i, d^(L-i)), the product in index 0 of every bond and zeros
 * elsewhere (Sec. 2.1 MPS; the padding reading is stated in the design notes).
 * site_vectors: complex [L][d], host. Errors: TEVO_EINVAL, TEVO_ENOMEM.
 */
int mps_init(tevo_ctx ctx, int L, int d, int D, const double* site_vectors, tevo_mps* out);
/* bond dimensions D_0..D_L (host array of L+1 ints) */
int mps_bond_dims(tevo_mps psi, int* dims_out);
/* copy site i's tensor A_i[D_{i-1}][d][D_i] to/from host (complex).
 * mps_set_site marks the state as not canonical. */
int mps_get_site(tevo_mps psi, int i, double* host_out);
int mps_set_site(tevo_mps psi, int i, const double* host_in);
/* accumulated log of the norm removed by the normalisation of each time step */
int mps_log_norm(tevo_mps psi, double* out);
int mps_destroy(tevo_mps psi);

/*
 * evolve_step -- one time step psi <- W psi / ||W psi||, fitted at psi's bond
 * dimensions by variational sweeps (Sec. 2.2 and Table 1, "(i)DMRG" row; the
 * set-up of Sec. 8.2: one variational fit per time step at fixed bond
 * dimension).
 *
 * The step starts from phi = psi (right-canonical), builds the right
 * environments of <phi|W|psi>, and runs `sweeps` sweeps (sites 1..L-1 moving
 * right with a Householder QR re-gauge, then sites L..2 moving left as the same
 * step on the mirrored chain), then recomputes the centre at site 1, normalises
 * it and accumulates log ||.|| in the state's log-norm.
 * tau must equal the tau W was built with (TEVO_ETAU otherwise); D must equal
 * the cap psi was created with (TEVO_ESHAPE otherwise). precision is one of
 * TEVO_FP64 / TF32 / TF32X3 / BF16X3: for the low-precision forms the first
 * sweeps-1 sweeps use tensor-core contractions and the last sweep (preceded by
 * a rebuild of the right environments) is fp64 (with sweeps = 1 the step is all
 * fp64); OR-ing TEVO_TC_ONLY makes every sweep a tensor-core sweep, OR-ing
 * TEVO_OZAKI computes the fp64 contractions with the tensor-core Ozaki scheme
 * (TEVO_OZAKI with TEVO_TC_ONLY is TEVO_EINVAL); OR-ing TEVO_TWO_SITE (with
 * TEVO_FP64, optionally TEVO_OZAKI) fits pairs of neighbouring sites instead of
 * single sites. The QR, the norm and every reduction are fp64 in all forms.
 * Errors: TEVO_EINVAL, TEVO_ESHAPE, TEVO_ETAU, TEVO_ENOMEM, TEVO_ECUDA,
 * TEVO_ENONFINITE (norm of the fitted state is 0, NaN or Inf), TEVO_ETIMEOUT
 * (a bounded device wait gave up), TEVO_EUNSUPPORTED. The work is issued on
 * the context stream; the call then synchronises to read the device status flags.
 */
int evolve_step(tevo_mps psi, tevo_mpo W, double tau_re, double tau_im, int D, int sweeps,
                int precision);

/*
 * evolve_step_batched -- one time step of n independent chains (each with its
 * own MPO, using that MPO's tau and each state's own D), the batched form of
 * evolve_step. Same sweeps / precision for every chain; each chain's result is
 * exactly the one evolve_step would give it.
 * The chains run concurrently on internal worker streams forked from the first
 * state's context stream and joined back into it. The first calls are issued
 * directly and time three schedules (worker-stream counts, largest chain first);
 * once every chain is in right-canonical form and the schedule is chosen, a
 * step is captured into a CUDA graph (one per psi/phi buffer parity) and later
 * steps replay it. Handles must not be used from other streams meanwhile.
 * TEVO_OZAKI is not built for the batched form (TEVO_EUNSUPPORTED).
 * Errors: as evolve_step, for the first failing chain. Synchronises.
 */
int evolve_step_batched(tevo_mps* psis, const tevo_mpo* Ws, int n, int sweeps, int precision);

/*
 * measure_local -- <O_i> = <psi|O_i|psi>/<psi|psi> for every site i and each of
 * nops single-site operators (the local observables of Sec. 8.2), in any gauge.
 * The left transfer matrices are built site by site; for a state left by
 * evolve_step (right-canonical from site 1 on, d <= 4) each value is
 * sum_{s,t} O[s][t] rho_i[s][t] with the site density
 * rho_i[s][t] = sum conj(A_i[a][s][b]) (El_i A_i)[a][t][b], otherwise the right
 * transfer matrices are built as well and each operator is contracted in.
 * ops: complex [nops][d][d] host; out: complex [nops][L] host.
 * Errors: TEVO_EINVAL, TEVO_ENOMEM, TEVO_ECUDA. Synchronises the stream.
 */
int measure_local(tevo_mps psi, int nops, const double* ops, double* out);

/*
 * mps_overlap -- <a|b> of the stored (normalised) tensors, returned as
 * log|<a|b>| and arg <a|b> so that long chains neither overflow nor underflow
 * (the fidelity density of Eq. fid is log_abs / L). The transfer matrix is
 * rescaled at every site. a and b need the same L and d.
 * Errors: TEVO_EINVAL, TEVO_ESHAPE, TEVO_ENOMEM, TEVO_ECUDA. Synchronises.
 */
int mps_overlap(tevo_mps a, tevo_mps b, double* log_abs, double* phase);

/*
 * tevo_gemm -- the complex contraction primitive of the sweep on its own:
 * C[m][n] = sum_k A[m][k] B[n][k] for complex fp64 device arrays A [M][K],
 * B [N][K] (row-major, k contiguous) and C [M][N] (row-major), computed in the
 * given precision: TEVO_FP64 on the fp64 pipe, TEVO_FP64 | TEVO_OZAKI (or
 * TEVO_OZAKI_SLICES(G)) as exact digit-slice products on the tensor cores, the
 * others on the tensor cores (operands rounded/split into the precision's
 * planes, fp32 accumulation, fp64 result). Device pointers, aligned to 16 bytes; temporary device memory comes
 * from the context's allocator and is released before returning.
 * Errors: TEVO_EINVAL, TEVO_ENOMEM, TEVO_ECUDA, TEVO_ETIMEOUT. Synchronises.
 */
int tevo_gemm(tevo_ctx ctx, int precision, int M, int N, int K, const double* A, const double* B, double* C);

/*
 * tevo_gemm_noalloc -- tevo_gemm for callers that cannot allocate device
 * memory: a process whose device memory is entirely handed to a pre-sized pool,
 * or code that runs where an allocation may block, fail or is not permitted. It
 * computes the same product as tevo_gemm (same kernels) but allocates nothing:
 * no cudaMalloc / cudaFree and no call of the context's allocator. Its temporary
 * storage is one fixed array of TEVO_NOALLOC_SCRATCH_BYTES bytes in device
 * memory, created with the library and kept by every GPU that loads the library
 * until the process exits. The paper has no counterpart; this is a property of
 * the library, not of the method.
 *  - Limit: the operand planes plus at least one set of split-K partials must
 *    fit the array (bf16x3 / tf32x3 need about 8 / 16 bytes per element of A and
 *    B plus 8 bytes per element of C); larger shapes return TEVO_ESHAPE without
 *    touching the device. The split-K count may be lower than tevo_gemm's, so
 *    results can differ from tevo_gemm's in the last fp32 rounding.
 *  - The first call on a device looks up the array's device address (with that
 *    device current); make that first call before any stream capture.
 *  - Every call uses the same array and leaves its contents behind; the call
 *    clears what must start at zero. Calls whose GPU work overlaps -- on two
 *    streams, or from two host threads -- race on the array: serialise them.
 *  - The context's device must be the current device (else TEVO_EINVAL): the
 *    array's address differs per device.
 * Arguments and layouts as for tevo_gemm, except that precision is one of
 * TEVO_FP64, TEVO_TF32, TEVO_TF32X3 or TEVO_BF16X3: the Ozaki flag (and any
 * other flag bit) is refused with TEVO_EINVAL. Errors: TEVO_EINVAL, TEVO_ESHAPE,
 * TEVO_ECUDA, TEVO_ETIMEOUT. Synchronises the context stream.
 */
#define TEVO_NOALLOC_SCRATCH_BYTES (64u << 20)
int tevo_gemm_noalloc(tevo_ctx ctx, int precision, int M, int N, int K, const double* A, const double* B,
                      double* C);

/*
 * tevo_wait_selftest -- exercises the bounded device-side wait used by the
 * tensor-core kernels: one thread waits on a shared-memory barrier that nothing
 * completes, gives up after limit_ms (0 < limit_ms <= 5000) and records a code
 * in a device flag, which is copied to *code. Returns TEVO_ETIMEOUT when the
 * wait gave up (the expected outcome); the context stays usable.
 */
int tevo_wait_selftest(tevo_ctx ctx, double limit_ms, int* code);

/* name of an error code */
const char* tevo_strerror(int code);

/* number of kernels this library launched on the context since creation or the
 * last reset (host-side count of launches issued by the library) */
int tevo_launch_count(tevo_ctx ctx, long long* count, int reset);

/*
 * Event-timed kernel profile (diagnostics for the roofline figures). While
 * enabled, the library records a CUDA event pair on the context stream around
 * every launch of the kernel classes below, with the algorithmic flop and byte
 * count of that launch (from its shape: useful complex multiply-adds x 8 flops;
 * operand reads + output write once each). tevo_prof_read synchronises the
 * stream, returns the totals of one class since the last read of that class,
 * and clears them.
 */
#define TEVO_PROF_GEMM64 0   /* fp64 complex GEMM (main kernel, split-K partials included) */
#define TEVO_PROF_GEMMTC 1   /* tensor-core complex GEMM */
#define TEVO_PROF_QR 2       /* Householder factorisation of one matrix (all its column steps) */
#define TEVO_PROF_FORMQ 3    /* explicit thin Q */
#define TEVO_PROF_GEMMOZ 4   /* Ozaki-scheme complex GEMM (slice products + split-K sum) */
#define TEVO_PROF_OZSPLIT 5  /* row exponents and digit slices of the two Ozaki operands */
#define TEVO_PROF_CLASSES 6
int tevo_prof_enable(tevo_ctx ctx, int enable);
int tevo_prof_read(tevo_ctx ctx, int cls, double* ms_total, long long* launches, double* flops_total,
                   double* bytes_total);

#ifdef __cplusplus
}
#endif

#endif /* TEVO_H */
