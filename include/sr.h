/*
 * sr.h -- C ABI of the GB300 pf-FRG flow library (libsr.so).
 *
 * The library integrates the pseudofermion functional renormalization group flow of
 * Buessen, arXiv:2109.13317 ("The SpinParser software for pseudofermion functional
 * renormalization group calculations on quantum magnets") on one GPU: the flow of the
 * self-energy Sigma(w) and of the two-particle vertex Gamma^{mu nu}_{i1 i2}(s, t, u)
 * (Sec. 3, Eqs. frg:flowexplicit:1particle / frg:flowexplicit:2particle) in the cutoff
 * Lambda, with symmetry-reduced lattice storage (Sec. 4.1), frequency interpolation and
 * trapezoidal integration (Sec. 4.2), Euler stepping (Sec. 4.3) and the spin correlation
 * chi(k) (Sec. 3, Eqs. frg:correlation and frg:structurefactor).
 *
 * Conventions
 *   - Every function returns an sr_status; SR_OK = 0.  On error, sr_last_error() returns a
 *     thread-local message.  No C++ exception crosses this boundary.
 *   - Host arrays passed in are caller-owned and only read during the call.
 *   - Device pointers (marked "device") are borrowed for the call; they must be valid
 *     allocations on the current device, ordered on the flow's stream.
 *   - The library owns all its internal device memory (sr_flow_destroy releases it).
 *   - An sr_flow is not thread-safe; use one per host thread.
 *
 * Readings of points the paper leaves open are fixed identically here and in the test
 * oracle: Sigma = -i gamma with gamma real and odd (so G(w) = 1/(i(w + gamma(w))));
 * theta(0) = 1 in the delta-point terms of the single-scale propagator; trapezoid nodes at
 * {+-w_n} plus the propagator break points, clipped to [-w_max, w_max]; interpolation
 * corners below the s = u diagonal read through the s <-> u relation.
 *
 * State layout (device, FP64), as in Sec. 4.4 of the paper with the site index fastest:
 *   sigma: gamma(w_n), n = 0..N-1 (Sigma(w_n) = -i gamma(w_n)).
 *   gamma: index ((pair(s_i, u_i) * N + t_i) * n_c + c) * N_s + r
 *          with pair(s, u) = s (s + 1) / 2 + u for s >= u (the stored octant),
 *          c = spin component (SU2: 0 = density Gamma^00, 1 = spin Gamma^zz;
 *          XYZ: 0 = Gamma^00, 1..3 = Gamma^xx, Gamma^yy, Gamma^zz;
 *          TRI: c = mu * 4 + nu for all 16 basis functions, stored as real g^{mu nu} with
 *          Gamma^{mu nu} = i g^{mu nu} for the six functions with exactly one of mu, nu = 0
 *          (the imaginary class of Eq. frg:parametrizationBasis2p), Gamma^{mu nu} = g^{mu nu}
 *          otherwise),
 *          r = symmetry-irreducible site (r = 0 is the reference site itself).
 *   N_entries = N (N + 1) / 2 * N * n_c * N_s.
 */
#ifndef SR_H_
#define SR_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SR_OK = 0,
    SR_EINVAL = 1,        /* invalid argument (checked on the host before any launch) */
    SR_ENOMEM = 2,        /* host or device allocation failed */
    SR_ECUDA = 3,         /* a CUDA runtime call failed */
    SR_ESYMMETRY = 4,     /* not all lattice sites are equivalent under the model's symmetries */
    SR_ENONFINITE = 5,    /* the flow produced NaN / Inf */
    SR_ETIMEOUT = 6,      /* a bounded device-side wait gave up */
    SR_EUNSUPPORTED = 7   /* valid request that this build does not implement (e.g. tensor cores on a TRI flow) */
} sr_status;

typedef enum { SR_SU2 = 0, SR_XYZ = 1, SR_TRI = 2 } sr_backend;
typedef enum { SR_FP64 = 0, SR_FP32_MIXED = 1 } sr_precision;
typedef enum {
    SR_EULER = 0,         /* one Euler step to lambda_next (Sec. 4.3) */
    SR_RK_ADAPTIVE = 1,   /* embedded Dormand-Prince 5(4) steps with error control to lambda_next */
    SR_RK_FIXED = 2       /* exactly one Dormand-Prince 5(4) step of size lambda_next - lambda */
} sr_method;

/* Lattice bond (Sec. 5.3): basis site `from_basis` of a cell to basis site `to_basis` of
 * the cell shifted by da[0] a0 + da[1] a1 + da[2] a2. */
typedef struct { int from_basis, to_basis; int da[3]; } sr_bond;

/* Spin interaction (Sec. 5.4): S_from . M . S_to between sites given as (n0, n1, n2, basis);
 * M is row-major and already multiplied by the coupling constant. */
typedef struct { int from[4]; int to[4]; double M[3][3]; } sr_coupling;

typedef struct {
    double prim[3][3];             /* prim[i] = Cartesian lattice vector a_i */
    int n_basis;
    const double* basis_xyz;       /* host, n_basis x 3 Cartesian basis positions */
    int n_bonds;
    const sr_bond* bonds;          /* host */
    int n_couplings;
    const sr_coupling* couplings;  /* host */
    int range_L;                   /* truncation range in bonds (Sec. 4.1) */
    sr_backend backend;            /* SR_SU2 (Heisenberg), SR_XYZ (diagonal J) or SR_TRI (any J) */
    double eps;                    /* real-space precision of the symmetry search; <= 0 means 1e-5 */
} sr_lattice_desc;

typedef struct sr_lattice sr_lattice;
typedef struct sr_flow sr_flow;

/* Build the truncated lattice and its symmetry tables on the host (Sec. 4.1): the sites
 * within bond distance L of the reference site (basis site 0 of cell 0), the lattice and
 * spin-permutation symmetries of the model, the irreducible site set, the site-exchange
 * map, and the lattice-sum table of sum_j Gamma_{i1 j} Gamma_{j i2}.  The TRI core (Sec. 3,
 * the general time-reversal-invariant case) combines lattice symmetries with the 24 proper
 * rotations among the signed permutations of x, y, z.  No GPU is touched.
 * Errors: SR_EINVAL (bad desc), SR_ESYMMETRY (sites not all equivalent),
 * SR_EUNSUPPORTED (a coupling the chosen core cannot represent: off-diagonal J outside
 * TRI, anisotropic J in SU2). */
sr_status sr_lattice_create(const sr_lattice_desc* desc, sr_lattice** out);

/* N_s irreducible sites, N_tot sites within range, basis size, P lattice-sum table length. */
sr_status sr_lattice_info(const sr_lattice* lat, int* N_s, int* N_tot, int* N_basis, long* P);

/* Representative site (n0, n1, n2, basis) of each irreducible site: host out, N_s x 4. */
sr_status sr_lattice_representatives(const sr_lattice* lat, int* rep);

/* Map an arbitrary site pair (i1, i2) (each n0, n1, n2, basis) to the stored vertex:
 * *r = irreducible site or -1 if beyond range, perm[c] = stored component holding
 * component c of the pair (perm has 4 entries; for SU2 only c = 0, 1 are meaningful). */
sr_status sr_lattice_map_pair(const sr_lattice* lat, const int* i1, const int* i2, int* r, int* perm);

/* As sr_lattice_map_pair for every core, with signs: component c (c < n_c) of the pair
 * (i1, i2) equals sign[c] * stored component comp[c] of irreducible site *r (comp, sign:
 * host out, n_c entries each; n_c = 2, 4 or 16).  For SU2 / XYZ the signs are +1; for TRI
 * the map is a signed permutation of the 16 basis functions (Sec. 4.1 symmetries with a
 * spin rotation).  *r = -1 beyond range.  Errors: SR_EINVAL. */
sr_status sr_lattice_map_pair_components(const sr_lattice* lat, const int* i1, const int* i2, int* r, int* comp, int* sign);

sr_status sr_lattice_destroy(sr_lattice* lat);

/* Logarithmic frequency mesh w_n = w_min (w_max / w_min)^(n / (n_freq - 1)) (Sec. 5.2). */
sr_status sr_frequency_mesh_exponential(int n_freq, double w_min, double w_max, double* out);

/* Create a flow on the current CUDA device and the given stream (cudaStream_t, NULL =
 * default stream): initial condition Sigma = 0, Gamma^{mu nu} = J^{mu nu}/4 at
 * lambda_init (Sec. 3, Eq. frg:parametrizationInitial).  freq_pos: host, n_freq >= 2
 * strictly ascending positive frequencies.  Uploads the lattice tables. */
sr_status sr_flow_init(const sr_lattice* lat, int n_freq, const double* freq_pos, double lambda_init,
                       sr_precision precision, void* cuda_stream, sr_flow** out);

/* Number of stored Gamma entries and of frequencies. */
sr_status sr_flow_sizes(const sr_flow* flow, long* n_gamma, int* n_freq, int* n_comp);

/* Right-hand side of the flow at cutoff lambda for the current state: dgamma/dLambda
 * (device, N doubles) and dGamma/dLambda (device, N_entries doubles, state layout).
 * Either pointer may be NULL.  Asynchronous on the flow's stream. */
sr_status sr_flow_rhs(sr_flow* flow, double lambda, double* d_dsigma, double* d_dgamma);

/* Advance the state from the current cutoff toward lambda_next (< current) with the given
 * method; rtol / atol are the error-control tolerances of SR_RK_ADAPTIVE.  Writes the
 * cutoff reached to *lambda_reached (host; may be NULL).  Synchronises the stream once
 * per accepted or rejected step to read the error norm and the non-finite flag.
 * Errors: SR_EINVAL, SR_ENONFINITE (state untouched beyond the failing step). */
sr_status sr_flow_step(sr_flow* flow, double lambda_next, int method, double rtol, double atol,
                       double* lambda_reached);

/* Right-hand side restricted to the stored (s, u) pairs pair_begin .. pair_end - 1, the unit
 * of work the paper distributes over compute nodes (Sec. 4.4: all t, components and sites of
 * one (s, u) pair form a superblock), for flows sharded over several GPUs that all hold the
 * whole state.  dgamma/dLambda of every frequency goes to d_dsigma (device, N doubles; each
 * GPU recomputes it instead of broadcasting it); dGamma/dLambda of the pairs' entries goes to
 * d_dgamma (device, state layout) at their own positions, entries ((p N + t) n_c + c) N_s + r
 * for pair_begin <= p < pair_end, one contiguous slice; the rest of d_dgamma is not written.
 * Asynchronous on the flow's stream.  Errors: SR_EINVAL (range outside [0, N (N + 1) / 2],
 * null outputs). */
sr_status sr_flow_rhs_pairs(sr_flow* flow, double lambda, int pair_begin, int pair_end, double* d_dsigma,
                            double* d_dgamma);

/* Euler step (Sec. 4.3) with a right-hand side supplied by the caller, e.g. assembled from the
 * slices of several GPUs: y <- y - (lambda - lambda_next) f, f = (d_dsigma, d_dgamma) (device,
 * state layout); the cutoff becomes lambda_next.  Synchronises once (non-finite check).
 * Errors: SR_EINVAL (lambda_next outside (0, lambda)), SR_ENONFINITE. */
sr_status sr_flow_advance(sr_flow* flow, double lambda_next, const double* d_dsigma, const double* d_dgamma);

/* Largest number of attempted steps one SR_RK_ADAPTIVE call may take (default 10^6); when it
 * is exceeded the call returns SR_ETIMEOUT with the state and *lambda_reached at the last
 * accepted step. */
sr_status sr_flow_set_step_limit(sr_flow* flow, long max_steps);

/* Error norm of the last Dormand-Prince step, normwise:
 * max_i |e_i| / (atol + rtol max_i max(|y_i|, |y'_i|)),
 * and the counts of right-hand-side evaluations, accepted and rejected steps. */
sr_status sr_flow_stats(const sr_flow* flow, double* last_err, long* n_rhs, long* n_accept, long* n_reject);

/* Correlations at the current cutoff (Sec. 3, Eq. frg:correlation):
 * chi_ij (device, may be NULL): chi^{cc}_{b j} for every basis site b and site j within
 * range of b, layout [b][j][c], j in the order of sr_flow_chi_sites;
 * chi_k (host, may be NULL): structure factor (Eq. frg:structurefactor)
 * (1/N_b) sum_b sum_j cos(k (r_b - r_j)) sum_{mu = x,y,z} chi^{mu mu}_{b j} at the n_k
 * momenta k_xyz (host, n_k x 3).  Synchronises the stream when chi_k is requested. */
sr_status sr_measure_susceptibility(sr_flow* flow, int n_k, const double* k_xyz, double* chi_k,
                                    double* chi_ij);

/* Allocation-free variant of sr_measure_susceptibility, for callers that must not allocate
 * device memory while they run: hosts whose device memory is owned entirely by another
 * framework's pool or by a fixed budget, and code paths where a cudaMalloc (which may
 * synchronise the device or fail under memory pressure) is not acceptable.  It computes the
 * structure factor chi(k) of the current state into a caller-provided device array, reading
 * the momenta from a caller-provided device array; the intermediate chi_ij pair table is kept
 * in one file-scope device array of SR_CHI_STATIC_MAX doubles (2 MiB) that every GPU loading
 * the library holds until exit.  The paper has no counterpart to this entry point.
 *   d_k_xyz: device, n_k x 3 momenta;  d_chi_k: device, n_k outputs.
 * Requires N_basis x N_tot x n_comp <= SR_CHI_STATIC_MAX, else SR_EINVAL (nothing is launched
 * and d_chi_k is left untouched).  The flow's device must be the current device (SR_EINVAL
 * otherwise).  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before any stream
 * capture.  The call is asynchronous on the flow's stream and allocates nothing.  All calls
 * share the one array (each overwrites every entry it reads), so calls whose kernels overlap
 * on the GPU (different streams, no ordering between them) race and must be avoided. */
#define SR_CHI_STATIC_MAX 262144
sr_status sr_measure_susceptibility_static(sr_flow* flow, int n_k, const double* d_k_xyz, double* d_chi_k);

/* Site list used by chi_ij: for each basis b, the N_tot sites within range of b as
 * (n0, n1, n2, basis) (host out, N_basis x N_tot x 4). */
sr_status sr_flow_chi_sites(const sr_flow* flow, int* sites);

/* State access (device pointers, state layout).  get copies out, set copies in and sets
 * the current cutoff.  Either array may be NULL. */
sr_status sr_flow_get_state(const sr_flow* flow, double* d_sigma, double* d_gamma);
sr_status sr_flow_set_state(sr_flow* flow, double lambda, const double* d_sigma, const double* d_gamma);
sr_status sr_flow_lambda(const sr_flow* flow, double* lambda);

sr_status sr_flow_destroy(sr_flow* flow);

/* Lattice sum of an FP32-mixed SU2 flow on the tensor cores (off by default):
 * the per-triple contraction C_c[rA][rB] = sum over t-channel nodes of A[c][rA] B[c][rB]
 * (Eq. frg:flowexplicit:2particle, t-channel term with the site sum of Sec. 4.1) as tcgen05
 * MMAs in 3xTF32 (TF32 hi / lo splits of both operands, three products, FP32 accumulation in
 * tensor memory); off: the same contraction on FP32 CUDA cores.  SR_EUNSUPPORTED for FP64,
 * XYZ, or more than 64 padded irreducible sites. */
sr_status sr_flow_set_tensor_cores(sr_flow* flow, int on);
sr_status sr_flow_tensor_cores(const sr_flow* flow, int* on);

/* ---- tangent-linear flow: derivatives of the flow along coupling directions ---- */

/* Like sr_flow_init (FP64), but the state carries, with every value, its derivatives along
 * n_par <= 2 directions of the couplings: dM (host) holds n_par x n_couplings row-major
 * 3x3 matrices dM_c/dtheta_p in the order the couplings were given to sr_lattice_create.
 * The initial tangent is dJ/4 (Eq. frg:parametrizationInitial); every kernel then applies
 * the chain rule exactly (forward-mode dual numbers), so sr_flow_step (SR_EULER only)
 * integrates the tangent-linear flow beside the flow.  get/set_state and sr_flow_rhs see
 * interleaved (value, d/dtheta_1, d/dtheta_2) triples.  All three cores (SU2, XYZ, TRI; the
 * TRI kernel holds its rows as dual numbers in shared memory, so a TRI tangent flow takes
 * three times the shared memory of the FP64 flow).  Errors: SR_ESYMMETRY if a direction
 * is not invariant under the symmetries used to reduce the lattice (it could not be stored),
 * SR_EUNSUPPORTED if it has couplings the core cannot represent or the lattice needs more
 * shared memory than a CTA has. */
sr_status sr_flow_init_tangent(const sr_lattice* lat, int n_freq, const double* freq_pos, double lambda_init,
                               int n_par, const double* dM, void* cuda_stream, sr_flow** out);
sr_status sr_flow_tangents(const sr_flow* flow, int* n_tangent);

/* chi(k) and its derivatives d chi(k) / d theta_p of a tangent flow (host outputs: chi_k n_k,
 * dchi_k n_k x 2, p fastest).  Synchronises. */
sr_status sr_measure_susceptibility_tangent(sr_flow* flow, int n_k, const double* k_xyz, double* chi_k, double* dchi_k);

/* ---- adjoint (reverse mode) of the FP64 flow ----
 *
 * Transposed derivatives of the discretised flow of Sec. 3 / Sec. 4.2 (the same right-hand
 * side sr_flow_rhs evaluates) and of the Euler step of Sec. 4.3, for gradients of a scalar of
 * the final state (e.g. chi(k_max)) with respect to the initial state.  All three use the
 * flow's current state (set it with sr_flow_set_state: the caller keeps or recomputes the
 * forward trajectory, e.g. from checkpoints); none changes it.  Arrays are device pointers
 * on the flow's stream: sigma parts n_freq doubles, gamma parts n_gamma doubles (state
 * layout); outputs are overwritten; asynchronous except where noted.  All three cores (SU2,
 * XYZ, TRI).  Errors: SR_EUNSUPPORTED for FP32-mixed or tangent flows and when the lattice
 * needs more shared memory than one CTA has; SR_EINVAL for null pointers or a non-positive
 * cutoff.
 * Transposed lookups accumulate with atomic additions, so results are reproducible to
 * rounding, not bit for bit. */

/* (bar_sigma, bar_gamma) = (d f / d y)^T (fbar_sigma, fbar_gamma), f = sr_flow_rhs at lambda. */
sr_status sr_flow_rhs_adjoint(sr_flow* flow, double lambda, const double* d_fbar_sigma, const double* d_fbar_gamma,
                              double* d_bar_sigma, double* d_bar_gamma);

/* Adjoint of one Euler step y' = y - (lambda_from - lambda_to) f(lambda_from, y):
 * bar_out = bar_in - (lambda_from - lambda_to) (d f / d y)^T bar_in.  The flow's state must be
 * the forward state at lambda_from (SR_EINVAL otherwise).  Outputs may alias the inputs. */
sr_status sr_flow_step_adjoint(sr_flow* flow, double lambda_from, double lambda_to, const double* d_bar_sigma_in,
                               const double* d_bar_gamma_in, double* d_bar_sigma_out, double* d_bar_gamma_out);

/* Gradient of sum_i chi_bar_i chi(k_i) (sr_measure_susceptibility at the current state) with
 * respect to the state.  k_xyz (host, 3 n_k) and chi_bar (host, n_k) are copied; synchronises. */
sr_status sr_measure_susceptibility_adjoint(sr_flow* flow, int n_k, const double* k_xyz, const double* chi_bar,
                                            double* d_bar_sigma, double* d_bar_gamma);

/* Couplings linear in parameters theta: M_c = sum_p theta_p B_{p,c} for the n_couplings
 * interaction matrices of Sec. 5.4 (theta: host n_par; B: host n_par x n_couplings x 3 x 3
 * row-major; M: host out n_couplings x 3 x 3).  Errors: SR_EINVAL. */
sr_status sr_couplings_linear(int n_par, const double* theta, int n_couplings, const double* B, double* M);

/* Gradient of a scalar through the initial vertex Gamma_init = J / 4 (Sec. 3,
 * Eq. frg:parametrizationInitial): grad_p = sum over stored entries of (d Gamma_init /
 * d theta_p) bar_gamma, for coupling derivatives dM (host, n_par x n_couplings x 3 x 3 in the
 * order the couplings were given to sr_lattice_create; n_par <= 2) and the adjoint of the
 * initial state bar_gamma (device, state layout, e.g. from sr_flow_step_adjoint).  grad: host
 * out, n_par.  Synchronises.  Errors: SR_EINVAL; SR_EUNSUPPORTED for tangent flows and for
 * directions the core cannot represent (as sr_flow_init_tangent). */
sr_status sr_flow_initial_vertex_adjoint(sr_flow* flow, int n_par, const double* dM, const double* d_bar_gamma, double* grad);

/* ---- batched flows (many couplings / lattices of uneven size in one launch per stage) ---- */

typedef struct sr_batch sr_batch;

/* Group flows (all SR_FP32_MIXED, on the current device; the batch keeps pointers to them,
 * so they must outlive it).  The vertex flow of every instance runs in one persistent kernel
 * whose CTAs take (instance, stored triple) units from an atomic counter, largest instances
 * first; the paper's analogue is its dynamically balanced work units (Sec. 4.4).  TRI flows
 * (16 basis functions) run their own vertex kernel inside the batch's step; their self-energy
 * flow, integration nodes, update and FP32 copy share the batch's launches. */
sr_status sr_batch_create(int n, sr_flow* const* flows, sr_batch** out);

/* Integrate every flow with Euler steps (Sec. 4.3) through the common cutoff list
 * lambdas[0] > ... > lambdas[n_lambda-1] (host); every flow must be at lambdas[0].  With
 * use_graph != 0 one step is captured as a CUDA graph (the cutoff is read on the device from
 * the list) and replayed n_lambda - 1 times.  With autotune != 0 the node-block size and the
 * CTAs per SM of the persistent kernel are first chosen by timing every candidate on the
 * first step.  Synchronises; SR_ENONFINITE if any flow produced NaN / Inf. */
sr_status sr_batch_run(sr_batch* batch, int n_lambda, const double* lambdas, int use_graph, int autotune);

/* Chosen configuration (node-block size, CTAs per SM), its timed vertex-flow time (ms), the
 * device time of the last sr_batch_run (ms) and the number of work units per step. */
sr_status sr_batch_info(const sr_batch* batch, int* qc, int* ctas_per_sm, double* tune_ms, double* run_ms, long* units);

/* Size classes of the batch: instances are grouped by the shared memory their vertex flow
 * needs, and each class has its own persistent launch (CTAs per SM and node-block size
 * chosen by the autotuner).  sr_batch_class reports one class. */
sr_status sr_batch_classes(const sr_batch* batch, int* n_classes);
sr_status sr_batch_class(const sr_batch* batch, int k, int* n_instances, long* units, int* smem_bytes, int* qc,
                         int* ctas_per_sm, double* tune_ms);

/* Whether the classes' launches run as parallel graph branches (1) or one after another (0);
 * the autotuner times both and keeps the faster (parallel without autotuning). */
sr_status sr_batch_parallel_classes(const sr_batch* batch, int* parallel);

/* Launch form of the classes' vertex flow: mode 0 (default) lets the autotuner compare, per
 * class, the persistent kernel with the instances' own vertex kernels launched back to back
 * (as single flows launch them, here inside the batch's graph) and keep the faster; 1 forces
 * the persistent kernels, 2 the per-instance kernels.  Takes effect at the next sr_batch_run
 * (with autotune != 0 for mode 0).  Errors: SR_EINVAL (mode outside 0..2). */
sr_status sr_batch_force_launch(sr_batch* batch, int mode);

/* 1 if class k runs its instances' own kernels, 0 if its persistent kernel (host out). */
sr_status sr_batch_class_launch(const sr_batch* batch, int k, int* per_instance);

sr_status sr_batch_destroy(sr_batch* batch);

/* ---- measurement helpers (not part of the method) ---- */

/* Record CUDA events around every right-hand-side kernel launch on the flow's stream
 * (on != 0) or stop recording (on == 0, which also clears the record). */
sr_status sr_flow_profile_enable(sr_flow* flow, int on);

/* Recorded device time (ms) and launch count of the three right-hand-side kernels:
 * index 0 self-energy flow, 1 integration nodes, 2 vertex flow.  Synchronises. */
sr_status sr_flow_profile_read(sr_flow* flow, double* ms /*3*/, long* launches /*3*/);

/* Integration-node counts of the last right-hand side (host out, 3 x N: channel s, t, u
 * by transfer frequency), from which the algorithmic operation count follows.  Synchronises. */
sr_status sr_flow_node_counts(const sr_flow* flow, int* counts);

/* Number of distinct products in the lattice sum of one vertex entry (the deduplicated
 * pairs (stored site A, component) x (stored site B, component) over the table). */
sr_status sr_flow_lattice_sum_products(const sr_flow* flow, long* n_products);

/* Launch shape of the vertex kernels (host out, 4 ints): tensor-core kernel grid, its dynamic
 * shared memory, the runtime's occupancy figure for it, the CUDA-core kernel's shared memory. */
sr_status sr_flow_launch_info(const sr_flow* flow, int* info);

/* Throughput of fused multiply-adds on the current device (FLOP/s, 2 per FMA) for FP64
 * (precision = SR_FP64) or FP32 (SR_FP32_MIXED), from a register-resident FMA chain kernel
 * timed with CUDA events. */
sr_status sr_peak_fma(int precision, double* flops_per_s);

/* Thread-local message of the last error (empty string if none). */
const char* sr_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SR_H_ */
