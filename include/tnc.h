/*
 * tnc.h -- C boundary of the GB300 sliced tensor-network contraction library.
 *
 * The library computes amplitudes <x|U|0^n> of a quantum circuit by contracting its
 * tensor network (Sec. I; Sec. II-A: nodes are tensors, edges shared indices, each
 * pairwise contraction an M x K x N complex GEMM after permuting the common indices
 * to K; every index has dimension 2, Sec. III-A).  Slicing (Sec. II-A; Sec. III-A)
 * fixes s indices, giving 2^s independent subtasks whose sum is the amplitude.
 *
 * Conventions used by every call:
 *  - Status: every call returns tnc_status; TNC_OK on success.  No exception crosses
 *    the boundary.  tnc_last_error() returns a thread-local message for the last
 *    failure on the calling thread.
 *  - Ownership: handles are created by the library and released only by the matching
 *    tnc_*_destroy; every output buffer is allocated by the caller; the library never
 *    frees caller memory.  Device scratch belongs to a tnc_context and grows on demand
 *    (TNC_E_OOM when it cannot).
 *  - Bits: qubit q of an n-qubit register is bit (n-1-q) of a state index (qubit 0 is
 *    the most significant).  A bitstring is n bytes, byte q = bit of qubit q.
 *  - Gate matrices: row-major U[out, in], complex128 stored as interleaved (re, im)
 *    doubles, zero-padded to 4x4 (32 doubles).  For a 2-qubit gate on (q0, q1) the
 *    4-dim index is 2*bit(q0) + bit(q1).
 *  - Tensors handed to tnc_contract are "planar": a real plane of 2^rank values
 *    followed by an imaginary plane of 2^rank values; the element at flat index i
 *    has bit p of i equal to the value of the index labelled labels[p].
 *  - Asynchrony: calls that take a stream enqueue work and return; device-side
 *    failures (a bounded wait that ran out) surface at tnc_sync() as TNC_E_TIMEOUT.
 */
#ifndef TNC_H
#define TNC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t tnc_status;
enum {
  TNC_OK = 0,
  TNC_E_INVALID_ARG = 1, /* a pointer, size or option is out of range            */
  TNC_E_OOM = 2,         /* host or device allocation failed                      */
  TNC_E_CUDA = 3,        /* a CUDA call failed; message has the CUDA error string */
  TNC_E_TIMEOUT = 4,     /* a device-side bounded wait gave up                    */
  TNC_E_PLAN = 5,        /* the plan is inconsistent with the request             */
  TNC_E_UNSUPPORTED = 6, /* e.g. no sm_103 device, or a rank above the limits     */
  TNC_E_IO = 7           /* a plan file could not be read or written              */
};

/* Storage precision of the contraction path.  Arithmetic is FP32 in every case;
 * CHALF/CBF16 store tensors as fp16/bf16 planes with a power-of-two exponent per
 * tensor (exact scaling), C64 stores fp32 planes. */
enum { TNC_C64 = 0, TNC_CHALF = 1, TNC_CBF16 = 2 };

typedef struct tnc_circuit_s* tnc_circuit;
typedef struct tnc_network_s* tnc_network;
typedef struct tnc_plan_s* tnc_plan;
typedef struct tnc_context_s* tnc_context;

/* ---------------------------------------------------------------- circuit -> network */

/* Build a circuit from a gate list (Sec. I: the circuit that the network represents).
 *  n_qubits        1..64
 *  n_gates         >= 0
 *  arity[g]        1 or 2
 *  qubits[2*g+t]   qubit of slot t (t < arity[g]); distinct, in [0, n_qubits)
 *  matrices[32*g]  U[out, in] as above (host memory, copied)
 * Errors: TNC_E_INVALID_ARG on any out-of-range value. */
tnc_status tnc_circuit_from_gates(int32_t n_qubits, int64_t n_gates, const int32_t* arity,
                                  const int32_t* qubits, const double* matrices,
                                  tnc_circuit* out);
void tnc_circuit_destroy(tnc_circuit c);

/* A seeded random grid circuit of the family the paper simulates (Sec. I, Sec. VII): a
 * rows x cols grid, qubit q = r * cols + c; each of `cycles` cycles applies one single-qubit
 * gate per qubit, drawn from {sqrt(X), sqrt(Y), sqrt(W)} (each (I - i P)/sqrt 2, P = X, Y,
 * (X + Y)/sqrt 2) -- uniformly in the first cycle, then uniformly from the two that differ
 * from the qubit's previous gate -- then fSim(theta, phi) on the couplers of class A, B, C, D
 * in turn (A / B: horizontal pairs starting at even / odd columns; C / D: vertical pairs
 * starting at even / odd rows).  fsim_mode 0: theta = pi/2, phi = pi/6 everywhere; 1: both
 * uniform in [0, pi) per gate.  Gate order: a cycle's single-qubit gates by qubit, then its
 * fSim gates by coupler.  Draws come from splitmix64 streams seeded by `seed` (the gate
 * choices) and by seed ^ 0xD1B54A32D192ED03 (the angles).  Matrices as in
 * tnc_circuit_from_gates.  Errors: TNC_E_INVALID_ARG (grid outside 1..64 qubits, cycles < 0,
 * bad fsim_mode). */
tnc_status tnc_circuit_random_grid(int32_t rows, int32_t cols, int32_t cycles, uint64_t seed,
                                   int32_t fsim_mode, tnc_circuit* out);

/* The gates of a circuit in the layout tnc_circuit_from_gates reads (arity; qubits, -1 for
 * the unused second qubit; matrices as 32 doubles per gate, zero-padded), for an oracle or a
 * file.  n_qubits, n_gates: out (may be NULL).  With arity, qubits and matrices all NULL it
 * only reports the sizes; otherwise cap >= n_gates and any of the three may be NULL. */
tnc_status tnc_circuit_export(tnc_circuit c, int32_t* n_qubits, int64_t* n_gates, int32_t* arity,
                              int32_t* qubits, double* matrices, int64_t cap);

/* Build the tensor network of a circuit (Sec. II-A).  One tensor per 2-qubit gate with
 * its neighbouring 1-qubit gates multiplied in (a qubit without 2-qubit gates becomes
 * one rank-2 tensor); |0> inputs are fixed; output legs of qubits with
 * open_mask[q] != 0 stay open (the result is a tensor over them), the others are
 * fixed per bitstring at tnc_amplitudes time.
 *  open_mask  n_qubits bytes (host), or NULL for all closed. */
tnc_status tnc_network_build(tnc_circuit c, const uint8_t* open_mask, tnc_network* out);
void tnc_network_destroy(tnc_network n);

/* ---------------------------------------------------------------- order + slicing */

typedef struct {
  uint64_t seed;       /* seeds the Gumbel perturbation of the greedy order          */
  int32_t trials;      /* independent greedy trials; the cheapest total is kept      */
  int32_t log2_cap;    /* slice until every intermediate has at most 2^log2_cap entries */
  int32_t slices_min;  /* then add lowest-overhead indices up to this many (log2)    */
  int32_t slices_max;  /* trials above this many sliced indices are dropped if any  */
                       /* trial stays within it                                    */
  double temperature;  /* Gumbel temperature in log2-cost units; 0 = plain greedy    */
  int32_t mode;        /* 0: greedy pairwise order (balanced, "multi-stem" trees);     */
                       /* 1: stem order -- one tensor absorbs neighbouring leaves one  */
                       /*    at a time (the stem of Sec. II-A), which the fused chains */
                       /*    of Sec. IV execute on chip                               */
  int32_t objective;   /* which trial is kept: 0 = fewest complex multiply-adds (the    */
                       /* cost of Eq. 1); 1 = least modeled GB300 time of a call over   */
                       /* every slice: per step max(flops / rate, bytes / HBM bandwidth)*/
                       /* (tensor-core rate for steps large enough for its tiles) times */
                       /* the times it runs under tree-like reuse (Sec. III-B)          */
  int32_t slicing;     /* how the next sliced index is picked: 0 = smallest index     */
                       /* overhead O(a) of Eq. 1; 1 = lifetime-aware: smallest growth */
                       /* of the executed cost of all slices under tree-like reuse    */
                       /* (Sec. III-B), where an index costs only over the steps whose */
                       /* subtree fixes it.  With 1, objective 0 compares that cost.  */
  int32_t branch_exchange; /* 1: on the kept trial, exchange the order of two          */
                       /* consecutive contractions ((x g1) g2 -> (x g2) g1) while that */
                       /* lowers the cost the slicing uses and every intermediate     */
                       /* stays within the cap (Sec. III-C: nest sliced indices'      */
                       /* lifetimes); at most 8 passes                                */
  int32_t cluster_chains; /* 1: fused chains (Sec. IV) may hold tiles of up to 2^15     */
                       /* entries, spread over a thread-block cluster of up to 8 CTAs */
                       /* whose links read peers' shared memory (DSMEM); 0: one CTA, */
                       /* 2^12 entries                                                */
} tnc_plan_opts;

/* Greedy contraction order and slicing (Sec. II-A slicing; Sec. III-A, Eq. 1:
 * index overhead O(a) = 2 C_a / C_ori picks each sliced index).  Repeatedly contracts
 * the pair sharing an index that minimises size(out) - size(a) - size(b) (perturbed by
 * seeded Gumbel noise), then slices while an intermediate exceeds the cap, each time
 * taking the index of an oversized intermediate with the smallest O(a).  The result
 * holds the tree, the sliced indices and the compiled per-step program. */
tnc_status tnc_plan_greedy(tnc_network n, const tnc_plan_opts* opts, tnc_plan* out);
void tnc_plan_destroy(tnc_plan p);

typedef struct {
  double log2_flops_per_slice; /* log2 of complex multiply-adds of one slice           */
  double log2_total_flops;     /* log2 of complex multiply-adds of all 2^s slices       */
  double slicing_overhead;     /* 2^s * C_sliced / C_unsliced (Eq. 1 summed, Sec. III-A) */
  int32_t max_log2_size;       /* largest intermediate of one slice (log2 entries)      */
  int32_t n_sliced;            /* s                                                     */
  int32_t n_steps;             /* pairwise contractions per slice                       */
  int32_t n_leaves;
  int32_t n_open;              /* open output qubits (result has 2^n_open entries)      */
  int32_t n_kernels;           /* kernel launches per wave of instances (steps, leaf    */
                               /* gather, leaf scales, root sum; split steps add one)   */
  int32_t n_gemm, n_gepdot, n_absorb, n_fused; /* steps per class (a fused step counts */
                                               /* every contraction it contains)        */
  double narrow_max;           /* largest "narrow" rate 2 N_common / (N_A + N_B)       */
                               /* (Sec. VII-B) over the steps                          */
  double model_seconds_per_slice; /* modeled GB300 time of a call over every slice,    */
                               /* divided by 2^s (the objective = 1 cost; complex-half) */
  double log2_executed_flops;  /* log2 complex multiply-adds of all 2^s slices of one   */
                               /* bitstring under tree-like reuse (Sec. III-B)          */
  double log2_executed_flops_merged; /* the same with post-lifetime merging (Sec. III-B; */
                               /* tnc_exec_opts.reserved[1]): each sliced index summed    */
                               /* right after the step that contracts it                  */
} tnc_plan_info;
tnc_status tnc_plan_get_info(tnc_plan p, tnc_plan_info* info);

/* Statistics of each sliced index t (slice bit t; Sec. III-B lifetimes, Eq. 1 overheads),
 * at the plan's final slice set.  Any output pointer may be NULL; cap >= n_sliced.
 *  first_step, last_step  first / last step (in contraction order) whose operands hold
 *                         the index: its lifetime
 *  dep_steps              steps whose subtree fixes the index: they run once per value
 *                         of it under tree-like reuse
 *  overhead               2 C / C' with C the per-slice cost and C' that cost with t
 *                         unsliced (Eq. 1's index overhead, taken last)
 *  reuse_overhead         the same ratio of the executed cost of all slices under
 *                         tree-like reuse
 *  post_steps             dependent steps after the lifetime (they depend on the index
 *                         but no longer hold it)
 *  merge_saving           the fraction of that executed cost which summing over the
 *                         index right after its lifetime (post-lifetime merging,
 *                         Sec. III-B) would save: half of every post-lifetime step
 * Errors: TNC_E_INVALID_ARG (NULL plan, cap too small). */
tnc_status tnc_plan_slice_stats(tnc_plan p, int32_t* first_step, int32_t* last_step, int32_t* dep_steps,
                                double* overhead, double* reuse_overhead, int32_t* post_steps,
                                double* merge_saving, int32_t cap);

/* Sliced indices as wire segments: slice bit t (bit t of a slice id) fixes the wire of
 * qubit qubit[t] after cut[t] gates on that qubit.  cap >= n_sliced entries. */
tnc_status tnc_plan_sliced_cuts(tnc_plan p, int32_t* qubit, int32_t* cut, int32_t cap);

/* Open qubits in result order (first = most significant bit of the result index). */
tnc_status tnc_plan_open_qubits(tnc_plan p, int32_t* qubits, int32_t cap);

/* Replace the gate matrices of a plan's circuit (same gates, qubits and order; new values),
 * e.g. for a variational circuit.  The leaf tensors are re-formed on the host; the tree,
 * slices and compiled program are unchanged, and device programs re-upload the leaves
 * on their next use.  matrices: n_gates x 32 doubles as in tnc_circuit_from_gates. */
tnc_status tnc_plan_update_gates(tnc_plan p, int64_t n_gates, const double* matrices);

/* The whole plan as JSON text (network edges as [qubit, cut, kind, open], leaves with
 * their labels and gates, sliced edge ids, the tree as SSA pairs over tensor ids, every
 * tensor's labels in storage order and arena offset, the compiled steps with their
 * tiles; a tensor-core step also has "tc_tile": its row / column roles ("swap": rows from
 * operand b), tile width and depth and label sets).  Writes at most cap bytes including the terminating NUL; *len receives the
 * full size including the NUL, so a call with buf == NULL queries the size. */
tnc_status tnc_plan_describe(tnc_plan p, char* buf, int64_t cap, int64_t* len);

/* Plan persistence (binary, versioned).  The file holds the circuit, network, tree,
 * slices and options; loading recompiles the program. */
tnc_status tnc_plan_save(tnc_plan p, const char* path);
tnc_status tnc_plan_load(const char* path, tnc_plan* out);

/* ---------------------------------------------------------------- execution */

/* A context owns the device, its streams, the device program cache and scratch.
 * device: CUDA ordinal; the device must be sm_103 (GB300). */
tnc_status tnc_context_create(int32_t device, tnc_context* out);
void tnc_context_destroy(tnc_context ctx);

typedef struct {
  int32_t precision;     /* TNC_C64 / TNC_CHALF / TNC_CBF16                          */
  int32_t wave;          /* instances (bitstring x slice) contracted per launch; 0=auto */
  int32_t use_graph;     /* capture the per-wave launch sequence in a CUDA graph      */
  int32_t fuse;          /* 1 = fused on-chip chains of small absorptions (Sec. IV)  */
  int32_t profile;       /* 1 = time every step launch with CUDA events on the launch  */
                         /* stream; read with tnc_profile_read                        */
  int32_t reserved[3];   /* reserved[0], tnc_adjoint only: device memory (MiB) per instance
                            for the forward intermediates kept for the backward pass; above
                            it the largest are recomputed from their children when the
                            backward pass reaches them (0 = keep all).
                            reserved[1], tnc_amplitudes only: 1 = post-lifetime merging
                            (Sec. III-B, (sum_i A_i) B for sum_i A_i B): on a call over every
                            slice with tree-like reuse, the result of the step that contracts a
                            sliced index is summed over that index's two values right away,
                            so every later step runs half as often for it.  The sums
                            associate differently from the unmerged call (not bit-identical;
                            the same amplitudes within rounding).  Other calls ignore it.
                            reserved[2], tnc_amplitudes / tnc_amplitudes_ids: 1 = run each
                            wave's steps as one persistent launch (Sec. III-A: a wave's
                            subtasks in one launch) when every step of the program is a SIMT
                            contraction without merges: one cooperative kernel takes the steps
                            in order, its CTAs sharing each step's tiles, with a grid barrier
                            between steps.  Bit-identical to the per-step launches.  Other
                            programs, and profiled calls, run per step.
                            Others: 0. */
} tnc_exec_opts;

/* Amplitudes of a batch (Sec. I; the multi-amplitude batch of Sec. II-C), summed over
 * the slice ids [slice_begin, slice_begin + slice_count) (Sec. III-A: subtasks are
 * independent and their results add).  Slice id bit t fixes sliced index t; with 63 or
 * more sliced indices the ids address the slices whose indices 63 and up are 0.
 *  bitstrings  batch x n_qubits bytes (host); bits of open qubits are ignored.  May be
 *              NULL when batch == 1 and every qubit is open.
 *  out         batch x 2^n_open complex128 as interleaved (re, im) doubles; host or
 *              device memory (detected); entry (b, i) is the amplitude of row b with
 *              the open qubits set to the bits of i (first open qubit most significant).
 *  stream      cudaStream_t or NULL (the context's stream).  With a host `out` the
 *              call returns after the copy-back completes.
 * The cross-slice sum is accumulated in FP64 in a fixed order (deterministic). */
tnc_status tnc_amplitudes(tnc_context ctx, tnc_plan p, const tnc_exec_opts* opts,
                          const uint8_t* bitstrings, int64_t batch, int64_t slice_begin,
                          int64_t slice_count, double* out, void* stream);

/* The same sum over an explicit list of slice ids (a seeded subset of the slices, say): the
 * n_ids slices slice_ids[0..n_ids) (host array; each in [0, 2^s); a repeated id is counted
 * each time), added in list order.  Tree-like reuse does not apply.  Otherwise as
 * tnc_amplitudes.  Errors: TNC_E_INVALID_ARG (NULL or empty list, id out of range). */
tnc_status tnc_amplitudes_ids(tnc_context ctx, tnc_plan p, const tnc_exec_opts* opts,
                              const uint8_t* bitstrings, int64_t batch, const int64_t* slice_ids,
                              int64_t n_ids, double* out, void* stream);

/* Gradient environments (the derivative of L = sum_{b,i} w[b,i] * amp[b,i] with respect
 * to every gate matrix, holomorphic: dL/dU_g[o, i]).  Walks the contraction tree in
 * reverse: for a step C = A * B, dL/dA = contract(dL/dC, B) and dL/dB = contract(A,
 * dL/dC), the same pairwise contraction kind as the forward steps (Sec. II-A).
 *  weights  batch x 2^n_open complex128 interleaved (host)
 *  env_out  n_gates x 32 doubles (host): dL/dU_g as d x d row-major complex (d = 2 or 4) in
 *           the first d*d entries, the layout of the matrices of tnc_circuit_from_gates
 *  amp_out  optional (may be NULL): the amplitudes, as tnc_amplitudes
 * Computed in C64 (FP32) with the FP64 cross-slice accumulation, over every slice of the
 * plan (TNC_E_UNSUPPORTED above 30 sliced indices). */
tnc_status tnc_adjoint(tnc_context ctx, tnc_plan p, const tnc_exec_opts* opts,
                       const uint8_t* bitstrings, int64_t batch, const double* weights,
                       double* env_out, double* amp_out, void* stream);

/* One pairwise contraction C = A * B of planar binary-index tensors on the device
 * (Sec. II-A M x K x N view; Sec. V-A permutation folded into the loads; Sec. V-B
 * split over the common indices when M*N is small).  Labels are arbitrary int32
 * values; common labels are summed, C's labels must be the free labels of A and B.
 *  a, b, c    device pointers, planar, element type per precision (float, __half,
 *             __nv_bfloat16); c must not alias a or b.  2^rank entries per plane.
 *  ranks      0..32
 *  c_exp2     out (host): C's stored values times 2^(*c_exp2) are the result (inputs
 *             are taken at scale 1).
 * Errors: TNC_E_INVALID_ARG on inconsistent labels. */
tnc_status tnc_contract(tnc_context ctx, int32_t precision, const void* a, int32_t rank_a,
                        const int32_t* labels_a, const void* b, int32_t rank_b,
                        const int32_t* labels_b, void* c, int32_t rank_c,
                        const int32_t* labels_c, int32_t* c_exp2, void* stream);

/* The same single contraction as tnc_contract, for callers that cannot allocate device
 * memory: real-time threads that must not take the allocator's locks or wait on the
 * device synchronisations an allocation may imply, and applications whose own pool
 * allocator has already reserved the device's memory.  It takes no context and allocates
 * nothing: the scratch it needs (a few max/exponent slots and, for split-over-K shapes,
 * the FP32 partial sums) is one file-scope device array of 4 MiB that every GPU which
 * loads this library holds until the process exits.
 * There is no counterpart in the paper; this is an interface choice of this library.
 *  - Device: the caller's current device; a, b, c must live there.  The first call on a
 *    device looks up the array's device address (cudaGetSymbolAddress); make that first
 *    call before any stream capture.
 *  - Arithmetic: always the FP32 SIMT kernels (never the tensor-core kernel).
 *  - Limit: the split-K partials must fit in 4 MiB - 256 B.  A split step has at most
 *    2^10 outputs, and its split count is halved (each CTA then sums a longer K range)
 *    until splits x outputs x 8 B fits, so no contraction this library accepts needs
 *    more; the check that would reject a larger need with TNC_E_INVALID_ARG (the message
 *    gives the size) remains as a guard.
 *  - Sharing: every call uses the same array; the slots are cleared on each call, but
 *    calls that overlap on the GPU (several streams, or several host threads) race on it.
 *  - stream: cudaStream_t or NULL (the legacy default stream); the call copies C's
 *    exponent to the host and synchronises the stream, so it returns after C is ready.
 * Other arguments, layouts and errors are those of tnc_contract. */
tnc_status tnc_contract_noalloc(int32_t precision, const void* a, int32_t rank_a, const int32_t* labels_a,
                                const void* b, int32_t rank_b, const int32_t* labels_b, void* c,
                                int32_t rank_c, const int32_t* labels_c, int32_t* c_exp2, void* stream);

/* Per-launch timings of the last tnc_amplitudes call made with opts->profile = 1 on this
 * context, or of the last tnc_contract call (always timed: one entry, the contraction's
 * kernels without the two operand max passes; ms[1] the whole call) (waits for it).  Entry s is the s-th launch of the per-wave program (a step, or a
 * whole fused chain; cap >= n entries):
 *  ms[s]      device time summed over the call's launches of that step (CUDA events)
 *  launches[s] kernel launches of that step (per wave: 1, or 2 for a split step's reduce)
 *  flops[s]   algorithmic real flops of those launches: 8 * M * N * K per instance
 *  bytes[s]   algorithmic bytes: (|A| + |B| + |C|) * element size per instance
 *  kind[s]    kernel class (0 generic, 1 split-K GEPDOT, 2 fused chain, 3 tensor-core with
 *             cp.async gathers, 4 tensor-core with TMA loads, 5 persistent tensor-core
 *             with TMA loads: epilogue overlapped with the next tile's loads and MMAs,
 *             6 permute + tensor-core + permute (tnc_contract only), 7 GEPDOT streamed
 *             through a cp.async ring (split over K or not), 8 every step in one persistent
 *             launch (tnc_exec_opts.reserved[2]): entry 0 holds that launch's time and count,
 *             the other entries none)
 *  ms[n]      (one extra entry) the whole call's device time
 * *n receives the number of steps. */
tnc_status tnc_profile_read(tnc_context ctx, double* ms, int32_t* launches, double* flops, double* bytes,
                            int32_t* kind, int32_t cap, int32_t* n);

/* ---------------------------------------------------------------- autotuner */

/* Tile configurations of the tensor-core steps, chosen by timing (the step compiler's
 * configurations of Sec. IV and V, measured instead of predicted).  A tensor-core step's
 * admissible configurations are the ones its compiled operand layouts support:
 *  - tile widths of 256, 128 or 64 columns, at most the compiled width (a narrower tile
 *    loads a prefix of the compiled column labels; the rest become outer labels);
 *  - the persistent kernels (width <= 128 with two TMEM buffers; width 256 with the direct
 *    epilogue, one TMEM buffer handed back once drained into registers);
 *  - splits over the outer common labels, powers of two whose FP32 partial sums fit the
 *    program's partial-sum buffer;
 *  - a three-stage or a deep operand pipeline.
 * Every configuration computes the same contraction.  A different split changes only how
 * the FP32 partial sums are grouped.  For a fixed cache, results stay deterministic. */
typedef struct {
  int32_t steps_tuned;     /* tensor-core steps whose configurations were timed          */
  int32_t steps_changed;   /* steps now running a configuration other than the heuristics'*/
  int32_t candidates;      /* configurations timed                                       */
  int32_t reserved0;
  double seconds_default;  /* sum over the tuned steps of one launch, heuristic configs  */
  double seconds_tuned;    /* the same with the chosen configurations                     */
  double reserved[4];
} tnc_tune_info;

/* Runs tnc_amplitudes(ctx, p, opts, bitstrings, batch, slice_begin, slice_count) once,
 * discarding the result.  It then times the admissible configurations of every TMA
 * tensor-core step of the program that call used:
 *  - each at the call's wave size, on the call's stream;
 *  - one untimed launch, then 3 timed launches (23 when a launch is under 0.2 ms);
 *  - all configurations of a step in turn, three rounds, each keeping its fastest round.
 * A step takes the fastest configuration only if it beats the heuristics by 5% or more.
 * The choice is recorded in a process-wide cache keyed by the step's shape:
 *  - precision;
 *  - operand and result ranks;
 *  - compiled tile width and depth;
 *  - outer label counts;
 *  - epilogue kind;
 *  - instances per launch.
 * Programs built later take cached choices for steps of the same shape.  The tuned program
 * runs the chosen configurations from the next call on.
 *  info  may be NULL.
 * Errors: those of tnc_amplitudes.  Skipped without an error: C64 plans, and contexts
 * with TNC_NO_TC or TNC_NO_TMA set (they have no TMA steps). */
tnc_status tnc_autotune(tnc_context ctx, tnc_plan p, const tnc_exec_opts* opts,
                        const uint8_t* bitstrings, int64_t batch, int64_t slice_begin,
                        int64_t slice_count, tnc_tune_info* info);

/* The process-wide cache as a text file: the line "tnc-tune 1", then one line per shape:
 *   key bn persistent split stages
 *  - split: 0 means the heuristics;
 *  - stages: 0 heuristics, 1 deep, 3 three stages.
 * Save writes a temporary file and renames it into place.  Load merges the file's entries
 * into the cache; it changes nothing when any line is malformed.
 * Errors: TNC_E_INVALID_ARG (NULL path), TNC_E_IO (unreadable, unwritable or malformed).
 * Neither needs a GPU. */
tnc_status tnc_tune_save(const char* path);
tnc_status tnc_tune_load(const char* path);
void tnc_tune_clear(void);
int64_t tnc_tune_size(void);

/* Wait for the context's work and report device-side status (TNC_E_TIMEOUT if a
 * bounded wait ran out). */
tnc_status tnc_sync(tnc_context ctx);

/* Thread-local message of the last failure on this thread ("" if none). */
const char* tnc_last_error(void);

/* Library version string. */
const char* tnc_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TNC_H */
