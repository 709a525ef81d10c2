/*
 * qtpu_htn.h -- C ABI for contracting hybrid tensor networks (h-TNs) on one
 * NVIDIA B300 (sm_103a).
 *
 * What is computed (arXiv 2410.15080, section 4.1 and section 2.2): after the
 * quantum tensors (QTs) of a cut circuit have been evaluated into classical
 * tensors of subcircuit expectation values, the circuit's expectation value
 * <O> is the contraction of a tensor network made of those tensors and the
 * QPD coefficient tensors (CTs: a 6-vector per gate cut, the 4x4 tensor of
 * Eq. wire-tensor per wire cut).  An index shared by two or more tensors is
 * summed once (hyper-indices allowed, section 2.2); indices named as output
 * (for instance a batch of observables) are kept.  Section 4.2: the value
 * does not depend on the pairwise contraction order, the cost does; section
 * 6.1 steps 3 and 4 plan that order and then contract.
 *
 * Flow: create -> add_tensor (xN) -> set_output -> plan -> contract (xM).
 *
 * Ownership: tensor memory is BORROWED.  The caller keeps every device
 * buffer passed to add_tensor alive and unmodified until the stream work of
 * every contract call that reads it has completed.  The library owns its
 * plan, its device workspace and its status word; destroy frees them.  The
 * output is always FP64, written densely in the order of the output ids.
 *
 * Errors: every call returns a qtpu_status and nothing is thrown across the
 * ABI.  qtpu_last_error(h) returns a NUL-terminated message describing the
 * last failure on that handle (valid until the next call on it);
 * qtpu_last_error(NULL) describes the last failed call that takes no handle
 * (create, the allocation-free calls) on the calling thread.  A handle
 * is not thread-safe; the network is immutable after a successful plan.
 */
#ifndef QTPU_HTN_H
#define QTPU_HTN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct qtpu_htn qtpu_htn; /* opaque, library-owned */

typedef enum {
  QTPU_OK = 0,
  QTPU_EINVAL = 1,   /* bad argument: null pointer, rank/dim/stride/id error   */
  QTPU_ENOMEM = 2,   /* host or device allocation failed                      */
  QTPU_ECUDA = 3,    /* a CUDA runtime/driver call failed                     */
  QTPU_ESTATE = 4,   /* call out of order (e.g. contract before plan)         */
  QTPU_ETIMEOUT = 5, /* a bounded device-side wait gave up (status word)      */
  QTPU_ENOTSUP = 6,  /* unsupported (e.g. a size above 2^255, no GPU)         */
  QTPU_ELIMIT = 7    /* the peak-intermediate limit cannot be met by slicing  */
} qtpu_status;

typedef enum { QTPU_F32 = 0, QTPU_F64 = 1 } qtpu_dtype;

/* Arithmetic of the contraction.  With QTPU_PREC_FP64 every step runs in FP64
 * on the CUDA cores.  With a tensor-core precision:
 *   - the large pairwise GEMMs run on the tensor cores in the stated form with
 *     FP32 accumulation (BF16x3: pieces on a common grid per 64-entry k-block,
 *     so the leading-product accumulator of up to 1024 k is exact);
 *   - the other steps that produce intermediates (CT absorption, small or
 *     skinny contractions, operand gathers) compute in compensated FP32 pairs
 *     (hi + lo, about 44 significant bits) and store intermediates as pairs;
 *   - everything that produces values of the output accumulates in FP64 and
 *     writes FP64: the last step of every slice when it is a gather (the final
 *     dot product or reduction over signed QPD coefficients; a dot product
 *     folds pair sub-sums of at most 64 products into its FP64 accumulator),
 *     and the sum over slices, which reads a GEMM's (hi, lo) result exactly. */
typedef enum {
  QTPU_PREC_FP64 = 0,   /* every step in FP64 on the CUDA cores               */
  QTPU_PREC_TF32 = 1,   /* tensor cores, operands rounded to TF32 (1 product) */
  QTPU_PREC_3XTF32 = 2, /* tensor cores, 2-piece TF32 split, 3 products       */
  QTPU_PREC_BF16X3 = 3  /* tensor cores, 3-piece BF16 split, 6 products       */
} qtpu_prec;

/* informational for contraction (both kinds contract alike); QPD sampling
 * samples rank-1 CTs between two QTs (qtpu_htn_qpd_sample) */
typedef enum { QTPU_QT = 0, QTPU_CT = 1 } qtpu_kind;

typedef struct qtpu_plan_opts {
  uint64_t max_intermediate_bytes; /* 0 = no limit; 8 bytes per entry         */
  uint32_t n_slices;               /* minimum slice count; 0 or 1 = minimal   */
  uint32_t slice_dim;              /* only slice indices of this dim; 0 = any */
  qtpu_prec prec;
  int cost_model;                  /* 0 = exact FLOP cost; 1 = learned cost
                                      model (see qtpu_htn_plan)               */
  uint64_t seed;                   /* 0: greedy; else randomised greedy (the
                                      pair drawn among the 3 best keys by
                                      SplitMix64(seed)), for plan candidates */
  const char* autotune_table;      /* GEMM tile table file (see qtpu_htn_plan
                                      and qtpu_htn_autotune); NULL = the
                                      gemm_tiles_b300.txt next to the library
                                      if present; "" = none                   */
  uint32_t n_candidates;           /* > 1: plan with seeds seed, seed+1, ...,
                                      seed+n-1 (seed 0 = greedy) under the same
                                      slicing options and keep the plan with
                                      the fewest total FLOPs (ties: the lower
                                      seed); candidates that cannot meet the
                                      limit are skipped                      */
  uint64_t reuse_bytes;            /* sliced plans: device memory for
                                      intermediates with the copies slice
                                      reuse keeps (0 = 64 GiB, 1 = reuse
                                      off); see qtpu_htn_plan                 */
  const char* cost_model_path;     /* cost_model = 1: weights file (NULL =
                                      costmodel_b300.bin next to the library) */
  uint32_t search;                 /* order search (cost_model = 0 only):
                                      0 = greedy (best of n_candidates by
                                      plan FLOPs); 1 = hyper-search; 2 = the
                                      exact tree alone (see qtpu_htn_plan)    */
} qtpu_plan_opts;

/* Create an empty network bound to CUDA device `device` and the CUDA stream
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).  device = -1
 * creates a host-only handle that can plan and report its plan but not
 * contract (contract returns QTPU_ENOTSUP).  Fails with QTPU_EINVAL on a null
 * `out`, QTPU_ECUDA if the device cannot be selected. */
qtpu_status qtpu_htn_create(qtpu_htn** out, int device, void* cuda_stream);

/* Add one tensor (a QT or a CT; contraction treats both alike).
 *   rank       number of axes, 0..16
 *   index_ids  rank index ids (any int64 >= 0); an id names one index of the
 *              network; ids must be distinct within a tensor
 *   dims       rank extents, each >= 1; every occurrence of an id must have
 *              the same extent (else QTPU_EINVAL)
 *   dtype      QTPU_F32 or QTPU_F64
 *   dev_ptr    device pointer to the data (borrowed, see Ownership); may be
 *              NULL on a host-only handle
 *   strides    rank element strides (>= 0), or NULL for C row-major
 *   tensor_id  receives the tensor's id (0, 1, 2, ... in call order); may be
 *              NULL
 * QTPU_ESTATE after plan. */
qtpu_status qtpu_htn_add_tensor(qtpu_htn* h, qtpu_kind kind, int rank,
                                const int64_t* index_ids, const int64_t* dims,
                                qtpu_dtype dtype, const void* dev_ptr,
                                const int64_t* strides, int* tensor_id);

/* Name the output indices, in output order (n = 0: scalar output).  Every id
 * must occur on some tensor (checked by plan).  Default: scalar. */
qtpu_status qtpu_htn_set_output(qtpu_htn* h, int n, const int64_t* index_ids);

/* Plan the contraction (host only): greedy pairwise order on exact 256-bit
 * integer costs, then slicing until the peak intermediate fits
 * max_intermediate_bytes and the slice count reaches n_slices.  opts may be
 * NULL (defaults: no limit, no slicing, BF16X3, greedy).  QTPU_ESTATE with no
 * tensors, QTPU_EINVAL on an unknown output id, QTPU_ELIMIT if the limit
 * cannot be met, QTPU_ENOTSUP on a size of 2^255 or more.
 *
 * Slice reuse (sliced plans): a step's value depends only on the sliced
 * indices carried by the leaves below it, and not on those an earlier step
 * already contracted.  Every launch therefore runs once per value of the
 * sliced indices its inputs depend on; a step that contracts a sliced index
 * adds its result up over that index's values (compensated FP32 pairs, like
 * a K chunk of the tensor-core accumulation; the last step adds every value
 * into an FP64 partial), and its result is kept in one copy per value of the
 * sliced indices it still depends on.  Where those copies would exceed
 * reuse_bytes, some sliced indices are held fixed in an outer loop instead
 * (all of them: one slice at a time, the plan's own schedule).  The plan (its
 * text and FLOPs) is unchanged; qtpu_htn_exec_stats reports what a
 * contraction executes.  reuse_bytes = 1 turns reuse off.
 *
 * Learned cost model (cost_model = 1, device handles only): the planner makes
 * n_candidates plans (64 if n_candidates <= 1; seeds seed .. seed+n-1 under
 * the same slicing options), lowers each without device memory, and a small
 * perceptron (weights from cost_model_path, trained on this library's own
 * per-launch timings) predicts the device time of every launch of every
 * candidate on the device; the plan with the smallest predicted contraction
 * time among those whose executed FLOPs are within the model's stored factor
 * of the fewest is kept (the exact FLOP count bounds the model).  The plan
 * text is then that seed's plan with its search line.  The choice never
 * changes a computed value: every plan is contracted by the same kernels.
 * QTPU_EINVAL if the weights file is missing or invalid, QTPU_ENOTSUP on a
 * host-only handle.
 *
 * Order search (search = 1 or 2): the exact tree contracts every small leaf
 * (<= 256 entries: the CTs) first, in ascending id, into the lowest-id large
 * leaf sharing an index with it, then finds the cheapest contraction tree
 * over the tensors left (at most 16) by dynamic programming over subsets
 * with the planner's step cost (ties to the smallest subset as a bit mask),
 * emits it in post order and slices it like any plan; search = 2 returns it
 * (QTPU_ENOTSUP above 16 tensors, 128 indices or a cost of 2^126), and its
 * plan text ends with "search exact tensors=m".  search = 1 plans the exact
 * tree (when possible) and n_candidates randomised greedy orders (64 if
 * n_candidates <= 1) on the host cores in parallel, lowers each without
 * device memory and keeps the one whose launch list executes the fewest
 * FLOPs under slice reuse (ties: fewer plan FLOPs, then the exact tree, then
 * the lower seed); its plan text ends with "search hyper candidates=N
 * chosen=exact|seed:S executed_flops=F".  QTPU_EINVAL for search > 2 or
 * search with cost_model = 1.
 *
 * GEMM tiles: each tensor-core step (a batched GEMM of the step's batch, m,
 * n and k index groups, section 4.2) runs with the 128-row M tile along m
 * or along n and an N tile of 128, 112, 96, 80, 64 or 48 columns.  A step
 * whose consumer takes its result as split pieces from its epilogue keeps
 * the orientation that consumer needs and 128 columns.  Every other step
 * takes the entry of the tile table (autotune_table) for its problem
 * (prec, batch, m, n, k) when there is one, else the padding rule: the
 * fewest tiles weighted by N + 128 for a tile of N columns.  QTPU_EINVAL
 * if a given table cannot be read or has a malformed line.  The choice never
 * changes a computed value beyond rounding order. */
qtpu_status qtpu_htn_plan(qtpu_htn* h, const qtpu_plan_opts* opts);

/* Measure the GEMM tiles of this handle's lowered plan on CUDA device
 * `device` (-1: the handle's own; a host-only handle's lowered plan can be
 * timed on any device, without its tensors' data): for every tensor-core
 * step's problem, each valid orientation and N tile is timed (the median of
 * `reps` launches, 1..1000, after one warm-up) on synthetic operand pieces of
 * the step's shape and operand-pair count, in device memory this call
 * allocates and frees; the fastest choice per problem
 * is merged into the tile table file `table_path` (created if missing;
 * entries of other problems are kept) as lines
 *   prec batch m n k : swap bn ms ms_rule ms_base
 * (swap 1: m runs along the N tile; median milliseconds of the choice, of
 * the padding rule's choice and of 128-column tiles with m along M unless
 * m < 64; only the first seven fields are required when a table is read).
 * Plan another handle with autotune_table = table_path to use it.
 * *n_problems (may be NULL) receives the number of problems timed.  It
 * runs on a stream of its own and synchronises it; other work on the device
 * at the same time distorts the timings.  QTPU_ESTATE before plan,
 * QTPU_ENOTSUP for device -1 on a host-only handle, QTPU_EINVAL on a NULL or
 * empty path, bad reps, or an unreadable table, QTPU_ENOMEM / QTPU_ECUDA on
 * device errors, QTPU_ETIMEOUT if a timed GEMM's bounded wait gave up. */
qtpu_status qtpu_htn_autotune(qtpu_htn* h, int device, const char* table_path, int reps, int* n_problems);

/* Canonical plan text (order, index groups, per-slice sizes and FLOPs,
 * slices, totals).  Writes at most len bytes including the NUL; *needed (if
 * not NULL) receives the full length + 1.  QTPU_ESTATE before plan. */
qtpu_status qtpu_htn_plan_info(const qtpu_htn* h, char* buf, size_t len,
                               size_t* needed);

/* The lowered launch list, one line per kernel launch of one slice (kind,
 * fast or generic gather, operand count, shape, operands, destination, useful
 * FLOPs, algorithmic bytes), then the reduction and a summary line
 * (launches per slice, tensor-core steps, fused absorption steps, ...).
 * Available after plan, also on a host-only handle (lowering needs no GPU).
 * Same buffer convention as qtpu_htn_plan_info. */
qtpu_status qtpu_htn_lowering_info(const qtpu_htn* h, char* buf, size_t len,
                                   size_t* needed);

/* Number of FP64 entries of the output (product of output dims). */
qtpu_status qtpu_htn_output_size(const qtpu_htn* h, int64_t* n);

/* Useful FLOPs of the planned contraction (2 per multiply-add, all slices),
 * as a double; the number of pairwise steps and of steps that run on the
 * tensor cores (0 on a host-only handle); the device workspace the handle
 * owns (on a host-only handle: would own); and the number of kernel
 * launches one contract call makes.  Any pointer may be NULL. */
qtpu_status qtpu_htn_plan_stats(const qtpu_htn* h, double* flops_total,
                                int* n_steps, int* n_tensor_core_steps,
                                uint64_t* workspace_bytes,
                                int64_t* launches_per_contract);

/* What one full contract call executes: the useful FLOPs (2 per multiply-add)
 * after slice reuse, the same with every slice computed in full (the plan's
 * total), the extra device bytes that slice reuse uses for kept copies of
 * intermediates (beyond computing one slice at a time), and the kernel
 * launches.  Available after plan, also on a host-only handle.  Any pointer
 * may be NULL; QTPU_ESTATE before plan. */
qtpu_status qtpu_htn_exec_stats(const qtpu_htn* h, double* flops_executed,
                                double* flops_all_slices, uint64_t* kept_bytes,
                                int64_t* launches);

/* Features of every lowered launch for the learned cost model: row i (of
 * QTPU_N_LAUNCH_FEATURES floats, written to features + i * that count for
 * i < max_rows) describes launch i of the launch list (kind, work, shape,
 * tile fill, access pattern), launches[i] (may be NULL) how many kernel
 * launches of it one contraction makes; *n_rows receives the number of
 * launches.  Available after plan, also on a host-only handle. */
#define QTPU_N_LAUNCH_FEATURES 32
qtpu_status qtpu_htn_launch_features(const qtpu_htn* h, int max_rows, float* features,
                                     int64_t* launches, int* n_rows);

/* Kernel classes reported by qtpu_htn_profile_read. */
typedef enum {
  QTPU_K_CONTRACT = 0, /* FP64 pairwise step on the CUDA cores            */
  QTPU_K_SPLIT = 1,    /* operand gather + split into tensor-core pieces  */
  QTPU_K_GEMM = 2,     /* tcgen05 batched GEMM                            */
  QTPU_K_REDUCE = 3,   /* slice sum / final reduction                     */
  QTPU_K_COUNT = 4
} qtpu_kernel_class;

/* Enable (1) or disable (0) timing of every launch with CUDA events recorded
 * on the handle's stream around it.  Off by default. */
qtpu_status qtpu_htn_profile(qtpu_htn* h, int enable);

/* Wait for the stream, then return per kernel class (arrays of n entries,
 * n <= QTPU_K_COUNT, indexed by qtpu_kernel_class) the summed device time in
 * ms, the launch count, the useful FLOPs and the algorithmic bytes (each
 * operand read once, each result written once) of the launches timed since
 * the last read, and reset the counters.  Any array may be NULL. */
qtpu_status qtpu_htn_profile_read(qtpu_htn* h, int n, double* ms, int64_t* launches,
                                  double* flops, double* bytes);

/* Wait for the stream, then return every launch timed since the last read,
 * in order: launch_index[i] its index in the launch list (-1: the final
 * reduction) and ms[i] its device time; *n receives the count.  If max is
 * below the count nothing is written or reset (call again with room for *n
 * entries); otherwise the timings are reset like qtpu_htn_profile_read. */
qtpu_status qtpu_htn_profile_launches(qtpu_htn* h, int max, int* launch_index, double* ms, int* n);

/* Contract: enqueue the whole contraction on the handle's stream and write
 * the FP64 result (output_size entries) to the device buffer dev_out.
 * Asynchronous: returns after enqueueing.  Device-side failures (a bounded
 * wait that timed out) are reported by qtpu_htn_sync.  QTPU_ESTATE before
 * plan, QTPU_ENOTSUP on a host-only handle. */
qtpu_status qtpu_htn_contract(qtpu_htn* h, double* dev_out);

/* End-to-end form with HOST buffers: copies host_ptrs[t] (one per tensor,
 * dense row-major in the tensor's dtype, ideally pinned) into the device
 * buffers given to add_tensor, contracts, copies the FP64 result to host_out
 * (ideally pinned too: a pageable host_out makes the download a staged
 * synchronous copy, 0.3 ms on B300) and waits for the stream.  The uploads run on a copy stream of the handle,
 * in the order the contraction first reads the tensors, after the work
 * already enqueued on the handle's stream; each kernel waits only for the
 * uploads of the tensors it reads, so the contraction overlaps the later
 * uploads (its launches are direct, not the replayed graph).  Returns the
 * device status like qtpu_htn_sync. */
qtpu_status qtpu_htn_contract_host(qtpu_htn* h, const void* const* host_ptrs,
                                   double* host_out);

/* Contract n planned networks (of any shapes) and write dev_out[i] for each.
 * All n contractions run as ONE CUDA graph.  Small networks whose launches
 * are all gathers (unsliced, no tensor-core step, no launch above 2^16 terms)
 * can become tasks of one persistent kernel -- by default when they are at
 * least half of the batch (on B300, batches of 512 random networks in which
 * 52-80 % qualify ran 1.06-1.99x faster than as graph branches): its
 * blocks claim work
 * units (256 outputs of a launch, or
 * one output of a long sum) in task order, level by level across the
 * networks, and each unit first waits -- bounded by a time limit -- until the
 * same network's previous launch is complete.  The other networks' launches
 * form branches of the graph, spread over parallel streams (networks own
 * disjoint workspaces).  The graph is built on the first call for a given
 * (handles, outputs, options) list and replayed by later calls with the same
 * list; it is ordered after the work already enqueued on cuda_stream (NULL =
 * the first handle's stream), which waits for it.  Handles must be distinct
 * and share one device.  A wait of the persistent kernel that gives up marks
 * every network whose result it left incomplete: qtpu_htn_sync on that handle
 * returns QTPU_ETIMEOUT. */
qtpu_status qtpu_htn_contract_batch(qtpu_htn* const* hs, int n,
                                    double* const* dev_out, void* cuda_stream);

typedef struct {
  int persistent;            /* 2 (default): the persistent kernel for the
                                small gather-only networks when they are at
                                least half of the batch; 1: always for them;
                                0: graph branches only                       */
  uint64_t wait_limit_ns;    /* bound of the persistent kernel's dependency
                                waits; 0 = 2 s, at most 10 s                 */
  int test_stall_network;    /* test hook: >= 0 makes one dependency of that
                                network's tasks never complete, so its wait
                                gives up after wait_limit_ns; -1 = off        */
} qtpu_batch_opts;

/* qtpu_htn_contract_batch with options (opts NULL = the defaults). */
qtpu_status qtpu_htn_contract_batch_ex(qtpu_htn* const* hs, int n,
                                       double* const* dev_out, void* cuda_stream,
                                       const qtpu_batch_opts* opts);

/* For the most recent batch graph of this (handles, outputs) list: how many
 * networks the persistent kernel contracts and its task count.  QTPU_ESTATE
 * if no such graph exists. */
qtpu_status qtpu_htn_batch_info(qtpu_htn* const* hs, int n, double* const* dev_out,
                                int* n_persistent, int* n_tasks);

/* Contract only slices [first, first + count) of the planned contraction
 * (slices are the value assignments of the sliced indices, last sliced index
 * fastest) and write the FP64 sum of their results to dev_out.  The outputs
 * of disjoint ranges that cover [0, n_slices) add up to the full result, so a
 * long contraction can be split into resumable pieces or spread over devices.
 * Runs with direct kernel launches on the handle's stream.  QTPU_EINVAL on a
 * range outside [0, n_slices), QTPU_ENOTSUP for a network without pairwise
 * steps. */
qtpu_status qtpu_htn_contract_slices(qtpu_htn* h, int64_t first, int64_t count,
                                     double* dev_out);

/* Wait for the handle's streams and read its device status word: QTPU_OK, or
 * QTPU_ETIMEOUT if a bounded device-side wait gave up, or QTPU_ECUDA.  A
 * nonzero status is reported once (reading clears it). */
qtpu_status qtpu_htn_sync(qtpu_htn* h);

/* Failure-path self-test: enqueue on the handle's stream one warp whose
 * bounded device-side wait (the same bounded mbarrier wait the GEMM pipeline
 * uses) is on a barrier that nothing completes.  After limit_ns (at most 10
 * s) it gives up and sets the timeout bit of the status word, so the next
 * qtpu_htn_sync returns QTPU_ETIMEOUT.  Nothing faults, traps or hangs, and
 * the handle stays usable. */
qtpu_status qtpu_htn_selftest_timeout(qtpu_htn* h, uint64_t limit_ns);

/* Failure-path self-test of the tensor-core GEMM itself: enqueue on the
 * handle's stream one BF16x3 GEMM launch (256 x 128 x 64, on one CTA per
 * tile with pair = 0 or on a CTA pair with pair = 1) whose producer issues no
 * copies.  The MMA issuer's and the epilogue's bounded waits give up after
 * limit_ns (at most 10 s); the kernel lets nothing in flight, frees its TMEM
 * and returns, and the next qtpu_htn_sync returns QTPU_ETIMEOUT.  Nothing
 * faults, traps or hangs, and the handle stays usable.  QTPU_ESTATE before a
 * device plan, QTPU_EINVAL for a bad pair or limit. */
qtpu_status qtpu_htn_selftest_gemm_timeout(qtpu_htn* h, int pair, uint64_t limit_ns);

/* ---- QPD sampling and h-TN simplification (section 4.3; Step 1 of
 * section 6.1) ----
 * A gate-cut CT is a rank-1 tensor added with kind QTPU_CT whose index is
 * carried by exactly two QTs (kind QTPU_QT) and by no other tensor, and is
 * not an output index.  A group is the set of gate-cut CTs between the same
 * two QTs (tensor ids a < b); groups are ordered by (a, b), the CTs of a
 * group by tensor id.  Wire-cut tensors (rank 2) and every other tensor are
 * not sampled.
 *
 * qtpu_htn_qpd_groups: the number of groups of the network (works on
 * host-only handles). */
qtpu_status qtpu_htn_qpd_groups(const qtpu_htn* h, int* n_groups);

/* Sample the network into a new, unplanned network *out on the same device
 * and stream, with the same output indices:
 *  1. each group is fused: one CT over one new index (id = the largest id of
 *     the network + 1 + group number), its entries the tensor product of the
 *     group's CTs (the first CT's index slowest), products in FP64 left to
 *     right; in each of the two QTs the group's axes become one axis at the
 *     place of the first of them (groups applied in order);
 *  2. each fused CT c (length D) is sampled s_qpd times: draw j of group x
 *     takes u = dev_uniforms[x * s_qpd + j] (uniform in [0, 1), FP64, on the
 *     device, n_groups * s_qpd of them, read only during this call) and
 *     picks the first i with P_i > u * gamma, where P_i = |c_0| + ... + |c_i|
 *     is accumulated left to right in FP64 and gamma = P_{D-1} (the last
 *     nonzero entry if there is none); the sampled CT is
 *     c'_i = sign(c_i) * ((gamma * count_i) / s_qpd);
 *  3. values never drawn are dropped: the fused CT keeps the drawn values in
 *     ascending order, and both QTs are copied (dtype kept, C order)
 *     restricted to them.
 * The contraction of *out is an unbiased estimate of the source's.  Tensor
 * order of *out: the source's tensors other than the group CTs, in order
 * (untouched ones borrowed: the source's device memory must stay valid while
 * *out is used), then the fused CTs in group order.  *out owns the device
 * memory of its fused CTs and truncated QTs, taken from a per-device
 * stream-ordered pool of the library that keeps freed memory for the next
 * sampling (qtpu_htn_destroy returns it in stream order); the copies run on
 * the stream after this call returns, which waits only for the kept sizes
 * (one small device-to-host copy).  QTPU_EINVAL on s_qpd outside
 * 1..2^32 or NULL arguments, QTPU_ENOTSUP on a host-only handle, more than 8
 * CTs in a group or a fused length of 2^31 or more, QTPU_ENOMEM /
 * QTPU_ECUDA on device errors. */
qtpu_status qtpu_htn_qpd_sample(const qtpu_htn* h, uint64_t s_qpd, const double* dev_uniforms, qtpu_htn** out);

/* For a network made by qtpu_htn_qpd_sample: per group x < max, the fused
 * length before sampling and the number of values kept; *n_groups receives
 * the number of groups (0 for any other network). */
qtpu_status qtpu_htn_qpd_info(const qtpu_htn* h, int max, int64_t* dim_before, int64_t* dim_kept, int* n_groups);

/* Naive circuit knitting (Eq. knitting, section 2.1), the baseline the
 * contraction is measured against: dev_out (FP64, output_size entries, the
 * output in set_output order) receives, for each output entry, the sum over
 * every global instance -- every assignment of every non-output index, the
 * summed index ids in ascending order as one mixed-radix number, last
 * fastest -- of the product of one entry of every tensor (QTs and CTs),
 * products and sums in FP64, partial sums added in a fixed order.  The work
 * is the product of all summed dimensions times the output size (returned in
 * *n_instances as instances, may be NULL).  Works on any device handle,
 * planned or not; runs on the handle's stream and returns when the sum is
 * complete.  QTPU_ENOTSUP on a host-only handle, more than 32 tensors, 40
 * summed or 8 output indices, 4e18 instances or 65535 outputs or more. */
qtpu_status qtpu_htn_knit_naive(qtpu_htn* h, double* dev_out, double* n_instances);

/* The network's tensors: their number, and tensor t's rank, index ids, dims,
 * element strides, dtype, kind and device pointer (each output may be NULL;
 * the arrays need max_rank >= rank entries, else QTPU_EINVAL). */
qtpu_status qtpu_htn_num_tensors(const qtpu_htn* h, int* n);
qtpu_status qtpu_htn_tensor_info(const qtpu_htn* h, int t, int max_rank, int* rank, int64_t* index_ids,
                                 int64_t* dims, int64_t* strides, qtpu_dtype* dtype, qtpu_kind* kind,
                                 const void** dev_ptr);

/* ---- QT evaluation: a statevector simulator of subcircuit instances
 * (section 4.1: a subcircuit is a QT whose entries are its instances'
 * expectation values; section 6.2 Step 2 evaluates them -- here exactly, as a
 * mock QPU) ----
 * Qubit 0 is the most significant bit of a basis state's index. */
typedef enum {
  QTPU_OP_U1 = 0,       /* u: 2x2 unitary on q0, row-major (re, im) pairs      */
  QTPU_OP_CZ = 1,       /* CZ on q0, q1                                        */
  QTPU_OP_GATE_CUT = 2  /* on q0: the local operation of gate cut `cut` for its
                           index value g, factor `side` (0 first, 1 second) of
                           the CZ decomposition (section 2.1): side 0 takes
                           I, Z, M, M, e^{+i pi/4 Z}, e^{-i pi/4 Z} for g = 0..5,
                           side 1 takes I, Z, e^{+i pi/4 Z}, e^{-i pi/4 Z}, M, M;
                           each is followed by e^{-i pi/4 Z}; M is the signed Z
                           measurement rho -> P0 rho P0 - P1 rho P1            */
} qtpu_op_kind;
typedef enum {
  QTPU_CUT_GATE = 0,     /* dim 6: the index of one QTPU_OP_GATE_CUT          */
  QTPU_CUT_MEASURE = 1,  /* dim 4: the wire leaves at cut_qubit, measured in
                            A = I, Z, X, Y (the observable carries A there)    */
  QTPU_CUT_PREPARE = 2   /* dim 4: the wire enters at cut_qubit, prepared in
                            |0>, |1>, |+>, |i> before the first operation      */
} qtpu_cut_kind;
typedef struct {
  int kind;        /* qtpu_op_kind */
  int q0, q1;
  int cut, side;   /* QTPU_OP_GATE_CUT */
  double u[8];     /* QTPU_OP_U1 */
} qtpu_qop;
typedef struct {
  int n_qubits;            /* 1..15 */
  int n_ops;               /* 0..4096 */
  const qtpu_qop* ops;     /* host memory */
  int n_cuts;              /* 0..16: the QT's axes after the observable axis */
  const int* cut_kind;     /* qtpu_cut_kind per cut */
  const int* cut_qubit;    /* per wire cut its qubit (distinct); ignored for gate cuts */
  int n_obs;               /* 1..64 observables */
  const char* paulis;      /* n_obs * n_qubits characters I, X, Y, Z (observable
                              k on qubit q at k * n_qubits + q); I on measured
                              wire qubits */
} qtpu_qt_program;

/* Evaluate the QT of one subcircuit on CUDA device `device` and stream
 * cuda_stream: dev_out[k][v_0][v_1]... (FP64, C order, dims n_obs, then 6 or 4
 * per cut) = Re Tr(O_k' E_v(rho_0)), rho_0 the product of the prepared wire
 * states and |0> elsewhere, E_v the operations with cut values v, O_k' the
 * observable k with A_{v_c} on each measured wire qubit -- the layout
 * qtpu_htn_add_tensor takes for the QT with index ids (k, cut_0, cut_1, ...).
 * Pure-state simulation in FP64: a signed measurement is carried as its two
 * projected branches, added with sign -1 for outcome 1.  Each instance is one
 * thread block, its state in shared memory up to 12 qubits (in device memory
 * the call allocates beyond); results are deterministic.  Returns when the QT
 * is written; *n_instances (may be NULL) receives the number of instances.
 * QTPU_EINVAL on a malformed program (qtpu_last_error(NULL) says which
 * rule), QTPU_ENOMEM / QTPU_ECUDA on device errors. */
qtpu_status qtpu_qt_evaluate(int device, void* cuda_stream, const qtpu_qt_program* prog, double* dev_out,
                             double* n_instances);

qtpu_status qtpu_htn_destroy(qtpu_htn* h);

/* Message of the last failure on h (or, when h is NULL, of the calling
 * thread's last failed call that takes no handle: create and the
 * allocation-free calls).  Never NULL. */
const char* qtpu_last_error(const qtpu_htn* h);

/* ------------------------------------------------------------------------
 * Learned cost model (ranks candidate plans; never changes a computed value).
 * A 3-layer perceptron  h1 = relu(x W1 + b1), h2 = relu(h1 W2 + b2),
 * y = h2 W3 + b3  on plan features x (FP32), predicting log contraction time.
 * Weights are used in BF16, rounded from FP32 master copies; products are
 * accumulated in FP32; loss = mean squared error; optimiser = Adam.
 * Parameter layout (FP32): W1[in][hidden] b1[hidden] W2[hidden][hidden]
 * b2[hidden] W3[hidden] b3. */
typedef struct qtpu_mlp qtpu_mlp;

/* Create a model on `device`, enqueueing on `cuda_stream`; weights drawn
 * uniformly in +-sqrt(6 / fan_in) from SplitMix64(seed), biases 0. */
qtpu_status qtpu_mlp_create(qtpu_mlp** out, int device, void* cuda_stream,
                            int in_dim, int hidden, uint64_t seed);
qtpu_status qtpu_mlp_num_params(const qtpu_mlp* m, int64_t* n);
/* Copy the FP32 master parameters out (host_out) and/or in (host_in). */
qtpu_status qtpu_mlp_params(qtpu_mlp* m, float* host_out, const float* host_in);
/* dev_y[b] = model(dev_x[b]) for b < batch; dev_x is [batch][in] FP32. */
qtpu_status qtpu_mlp_forward(qtpu_mlp* m, const float* dev_x, int batch, float* dev_y);
/* Gradients of the MSE loss against targets dev_t (FP32, parameter layout)
 * copied to host_grads, and the loss to host_loss (either may be NULL). */
qtpu_status qtpu_mlp_gradients(qtpu_mlp* m, const float* dev_x, const float* dev_t,
                               int batch, float* host_grads, float* host_loss);
/* One Adam step (beta 0.9 / 0.999, eps 1e-8) with learning rate lr; the
 * batch loss before the step goes to host_loss (may be NULL). */
qtpu_status qtpu_mlp_train_step(qtpu_mlp* m, const float* dev_x, const float* dev_t,
                                int batch, float lr, float* host_loss);
qtpu_status qtpu_mlp_destroy(qtpu_mlp* m);

/* Bytes of the fixed device scratch array used by
 * qtpu_pairwise_contract_noalloc (held by every GPU that loads the library,
 * from first use until the process exits). */
#define QTPU_NOALLOC_SCRATCH_BYTES (32u << 20)

/* Allocation-free pairwise contraction.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory at call
 * time -- code running inside a memory pool or arena that another component
 * sized in advance, latency-critical loops where cudaMalloc / cudaFree would
 * synchronise the device or stall, and plain C callers that only hold device
 * pointers and no allocator.  It performs the computation of one
 * tensor-core step of qtpu_htn_contract, with every scratch buffer taken from
 * a fixed file-scope device array of QTPU_NOALLOC_SCRATCH_BYTES.
 *
 *   C[b][m][n] = sum_k A[b][m][k] * B[b][k][n]   for b < batch, m < M, n < N
 *
 *   A, B, C    device pointers, FP64, dense row-major ([batch][M][K],
 *              [batch][K][N], [batch][M][N]); A and B are read, C written;
 *              all owned by the caller
 *   cuda_stream  the stream the work is enqueued on (NULL = legacy default);
 *              the call is asynchronous, runs on the calling thread's current
 *              device, and uses BF16x3 tensor-core arithmetic (error about
 *              6e-8 relative, as the regular entry points)
 *
 * Scratch needed: at most 2304 + 6*batch*(M+N)*round_up(K,8) + 8*batch*M*N
 * bytes (the exact figure: qtpu_pairwise_noalloc_scratch_bytes); a call that
 * needs more than QTPU_NOALLOC_SCRATCH_BYTES returns QTPU_ELIMIT and does
 * nothing.  QTPU_EINVAL on NULL pointers or sizes < 1, QTPU_ECUDA if a CUDA
 * call fails.  The first call on a device resolves the scratch array's device
 * address (cudaGetSymbolAddress) for that device; make that first call before
 * any stream capture.  Every call shares the one array and leaves its
 * contents behind; calls whose GPU work overlaps in time race on it and must
 * be serialised by the caller.  The call returns once the work is enqueued:
 * a device-side failure (a bounded wait of the GEMM that gave up) is reported
 * by qtpu_noalloc_status, which a caller that needs to know C is valid calls
 * after the work.  qtpu_last_error(NULL) returns the message of the last
 * failed allocation-free call on the calling thread. */
qtpu_status qtpu_pairwise_contract_noalloc(const double* A, const double* B, double* C,
                                           int batch, int M, int N, int K,
                                           void* cuda_stream);

/* Exact scratch bytes qtpu_pairwise_contract_noalloc needs for these sizes
 * (compare with QTPU_NOALLOC_SCRATCH_BYTES).  QTPU_EINVAL on a NULL `bytes`
 * or sizes < 1.  Host only: touches no device. */
qtpu_status qtpu_pairwise_noalloc_scratch_bytes(int batch, int M, int N, int K,
                                                size_t* bytes);

/* Wait for cuda_stream and report the device status of the allocation-free
 * calls enqueued on the current device: QTPU_OK, QTPU_ETIMEOUT if a bounded
 * device-side wait of the GEMM gave up (C is then not valid), QTPU_ECUDA if
 * a kernel rejected its arguments or a CUDA call failed.  Reading clears the
 * status (a failure is reported once).  Allocates nothing: the status word
 * lives in the fixed scratch array and is copied into a host variable. */
qtpu_status qtpu_noalloc_status(void* cuda_stream);

/* Failure-path self-test of qtpu_noalloc_status: enqueue on cuda_stream one
 * warp whose bounded wait (the GEMM pipeline's bounded mbarrier wait) is on a
 * barrier that nothing completes; after limit_ns (at most 10 s) it gives up
 * and sets the timeout bit of the allocation-free status word, so the next
 * qtpu_noalloc_status returns QTPU_ETIMEOUT.  Nothing faults, traps or hangs.
 * QTPU_EINVAL on a limit of 0 or above 10 s. */
qtpu_status qtpu_noalloc_selftest_timeout(uint64_t limit_ns, void* cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* QTPU_HTN_H */
