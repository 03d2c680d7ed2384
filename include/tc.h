/*
 * tc.h -- exact directed-graph triad census on one NVIDIA B300 (sm_103a).
 *
 * The library implements the subquadratic triad census of the thesis
 * "Study and evaluation of an Irregular Graph Algorithm on Multicore and GPU
 * Processor Architectures" (arXiv 1603.02655): for every unordered vertex
 * triple of a strict digraph, count which of the 16 MAN isomorphism classes
 * its induced sub-digraph belongs to (Sec. 2.2).  The problem statement of
 * Sec. 2.2 fixes the interface: input a digraph G=[V,E] with an explicit
 * order n, output the Census array of 16 frequencies.
 *
 * Conventions for every call
 *   - Vertex ids are 0-based int32 in [0, n).  (The thesis reads 0- or
 *     1-based files, Sec. 5.1.1; a caller with 1-based ids subtracts 1.)
 *   - Self-loops are dropped and duplicate arcs collapse: the census is of
 *     the strict digraph the arcs describe.  Isolated vertices count in C(n,3).
 *   - n must be < 2^30 (ids are packed as id<<2 | 2-bit tag in 32 bits).
 *   - Every call returns a tc_status and never aborts the process; no C++
 *     exception crosses this boundary.  On failure, tc_last_error() returns a
 *     thread-local description of the most recent error.
 *   - "stream" is a cudaStream_t (NULL = the legacy default stream).  The
 *     caller owns every input and output buffer; the library copies inputs
 *     it keeps and never frees caller memory.
 *   - A tc_graph is owned by the library until tc_graph_free.  Calls on the
 *     same graph must not run concurrently (they share its work space).
 */
#ifndef TC_H
#define TC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tc_graph_s* tc_graph;

typedef enum {
    TC_OK = 0,
    TC_ERR_ARG = 1,         /* null pointer, negative size, unknown flag */
    TC_ERR_ID_RANGE = 2,    /* an arc endpoint outside [0, n) */
    TC_ERR_OOM = 3,         /* a device allocation failed; nothing is leaked */
    TC_ERR_CUDA = 4,        /* a CUDA runtime call failed (see tc_last_error) */
    TC_ERR_TIMEOUT = 5,     /* a bounded device-side wait ran out */
    TC_ERR_UNSUPPORTED = 6  /* n >= 2^30, sizes beyond a stated limit, no device */
} tc_status;

/* Census in MAN order: count[t] for t = 0..15 is the thesis's type t+1,
 * 003 012 102 021D 021U 021C 111D 111U 030T 030C 201 120D 120U 120C 210 300
 * (Sec. 2.2).  The 003 count is C(n,3) minus all others (Sec. 2.2, the
 * null-triad step) and is returned as a 128-bit value: count[0] holds its
 * low 64 bits and count003_hi its high 64 bits, so it stays exact for every
 * n < 2^30.  The other fifteen counts are exact as long as they are below
 * 2^64 (true whenever |dyads| * n < 2^64). */
typedef struct {
    uint64_t count[16];
    uint64_t count003_hi;
} tc_census_t;

/* Census by the 64 labelled triad codes (the non-isomorphic census of Sec.
 * 2.2: Fig. "Triad Code Algorithm" without its TriadTable step).  Code =
 * e(u,v) + 2e(v,u) + 4e(u,w) + 8e(w,u) + 16e(v,w) + 32e(w,v), where <u,v>
 * (u < v, adjacent) is the canonical dyad that counts the triad and w its
 * third vertex: a connected triad is counted by the dyad for which w passes
 * the canonical test of Fig. "Subquadratic Triad Census Algorithm"; a triad
 * with a single adjacent pair u < v has code e(u,v) + 2e(v,u) (the dyadic
 * term); code 0 is the null triad, C(n,3) minus all others, 128-bit like
 * tc_census_t (count[0] low, count0_hi high 64 bits).  Mapping the codes by
 * the isomorphism table gives tc_census_t. */
typedef struct {
    uint64_t count[64];
    uint64_t count0_hi;
} tc_census64_t;

/* Statistics of a built graph (per graph of a batched build). */
typedef struct {
    int64_t n;              /* vertices */
    int64_t arcs;           /* distinct arcs after dropping loops/duplicates */
    int64_t dyads;          /* connected (canonical) dyads |U| */
    int64_t mutual;         /* mutual dyads */
    int64_t asym;           /* asymmetric dyads */
    int64_t merged_entries; /* sum over canonical dyads of |N(u)|+|N(v)| = sum_v d_v^2 */
    int64_t max_degree;     /* largest undirected degree */
} tc_graph_stats_t;

/* Task binning of the merge path (Sec. 4.3.1: canonical-dyad tasks, cost
 * |N(u)|+|N(v)|-2, the uniform distribution).  TC_BIN_EXACT bins by the exact
 * task cost |S| = |N(u) u N(v) \ {u,v}| instead (the W3 workload of Sec. 4.3,
 * balanced by the non-uniform distribution of Sec. 4.3.2): a pass before the
 * task pass (k_union_entries, one binary search per entry of the shorter
 * list) computes it for every canonical dyad, and a task goes to the thread
 * bin when |S|+2 <= thr_thread, the warp bin when <= thr_warp.  It is the
 * ceiling of a one-number cost rule; its pass is timed apart
 * (tc_profile_t.ms_exact_cost, not in ms_total).  Graphs on the forward path
 * have no bins and ignore bin_mode. */
enum { TC_BIN_HEURISTIC = 0, TC_BIN_MLP = 1, TC_BIN_EXACT = 2 };

typedef struct {
    int32_t bin_mode;     /* TC_BIN_HEURISTIC (degree sum), TC_BIN_MLP or TC_BIN_EXACT */
    int32_t thr_thread;   /* tasks with |N(u)|+|N(v)| <= thr_thread: one thread each */
    int32_t thr_warp;     /* <= thr_warp (capped at 1024): one warp each;
                             larger tasks are split into tiles */
    int32_t chunk;        /* merge outputs per tile of a split task: 256..1024
                             for warp tiles, 256..3840 for CTA tiles */
    int32_t profile;      /* 1: time each kernel with CUDA events and keep the
                             task/bin counts (read with tc_census_profile);
                             the call then synchronises `stream` */
    int32_t split_cta;    /* 0: tiles of split tasks run one per warp;
                             1: one per 256-thread CTA */
    int32_t stream_max;   /* tasks above thr_warp whose shorter list has at most
                             stream_max entries are streamed by one warp; the
                             others are split into tiles.  Shorter lists of at
                             most 1024 entries are staged whole and run in the
                             main merge; longer ones ("hub" tasks) run in a
                             separate launch that stages them 1024 at a time */
    int32_t persistent;   /* 1: the whole merge phase is one persistent launch
                             whose warps pull streamed tasks, tiles, warp tasks
                             and thread tasks from four queues (requires
                             split_cta = 0) */
    int32_t hub_ratio;    /* a hub task (shorter list above 1024 entries, within
                             stream_max) is streamed when its longer list has at
                             least hub_ratio times as many entries as the
                             shorter one, else split into tiles; >= 0 (0 and 1
                             stream every hub task) */
    int32_t own_min;      /* a dyad whose higher-degree endpoint (its owner; equal
                             degrees: the larger id) has degree d_h with
                             own_min <= d_h <= 131072 is not merged: the
                             owner's list is indexed by id buckets in shared
                             memory (and copied there up to 512 entries) and
                             the other endpoint's list is looked up in it.
                             0 disables; default 128 */
    int32_t row_tasks;    /* 1: compute the per-dyad terms with one warp per row
                             (the path used anyway when a row has 2^21 or more
                             entries); 0: one thread per adjacency entry */
    int32_t tri_path;     /* how the shared neighbours of the dyads (the
                             triangles) are found:
                             TC_TRI_FORWARD (0): each triangle once,
                             from degree-ranked forward lists (vertices ranked
                             by (floor(log2 degree), id); a dyad's owner is its
                             higher-ranked endpoint);
                             TC_TRI_MERGE (1): per-dyad owner lookups and merge
                             bins, tuned by the fields above (own_min,
                             thr_thread, thr_warp, chunk, stream_max, hub_ratio,
                             persistent, split_cta, bin_mode);
                             TC_TRI_AUTO (2, default): each graph takes the
                             path its router picks (tc_path_route): the
                             installed path model, else the degree-skew rule */
    int32_t fwd_big;      /* TC_TRI_FORWARD: owners with at least fwd_big forward
                             neighbours, or at least fwd_big / 8 of them and
                             at least 128 owned dyads (and at most 1024
                             forward neighbours and 2^17 vertices ranked above
                             them), get a CTA and an exact tag map of their
                             forward list in shared memory; the others a
                             binary search per lookup.  >= 1; default 64 */
} tc_opts;

enum { TC_TRI_FORWARD = 0, TC_TRI_MERGE = 1, TC_TRI_AUTO = 2 };

/* Per-kernel timing and binning of the calling thread's most recent
 * tc_census / tc_census_batched call made with opts.profile = 1. */
typedef struct {
    float ms_tasks;          /* task build + suffix-count terms (k_tasks) */
    float ms_split;          /* chunk start partitions (k_split) */
    float ms_tiles;          /* tiles of split tasks (k_warp or k_cta) */
    float ms_stream;         /* streamed tasks (k_stream); with persistent = 1
                                only the hub tasks */
    float ms_owner;          /* owner lookups (k_owner alone) */
    float ms_warp;           /* whole tasks, one warp each (k_warp) */
    float ms_thread;         /* thread-per-task merges (k_thread) */
    float ms_merge;          /* the whole merge phase (all merge kernels, or k_merge) */
    float ms_fold;           /* 64->16 fold and 003 closure (k_fold) */
    float ms_total;          /* first to last kernel */
    int32_t launches;        /* kernels launched by the call */
    int64_t bin_tasks[4];    /* dyads per bin: thread, warp, split into tiles, streamed */
    int64_t bin_entries[4];  /* merged entries |N(u)|+|N(v)| per bin */
    int64_t chunks;          /* tile records of split tasks */
    int64_t hub_tasks;       /* streamed tasks whose shorter list exceeds 1024
                                (counted in bin_tasks[2]) */
    int64_t hub_entries;     /* their merged entries (part of bin_entries[2]) */
    int64_t owner_items;     /* owner work items (pieces of up to 1024 list
                                positions) */
    int64_t owner_tasks;     /* dyads it handled (in no bin) */
    int64_t owner_entries;   /* their |N(u)|+|N(v)| */
    int64_t owner_probes;    /* lookups: entries of the non-owner endpoints'
                                lists above max(u, v) */
    int64_t owner_staged;    /* owner-list entries staged */
    /* TC_TRI_FORWARD (the merge-path fields above are then zero): */
    float ms_forward;        /* vertex ranks, forward lists and dyad records */
    float ms_tri_map;        /* lookups of tag-map owners (k_tri_big) */
    float ms_tri_search;     /* lookups of the other owners (k_tri_small) */
    float ms_owner_prep;     /* TC_TRI_MERGE: the owner dyads' lookup ranges
                                (k_owner_prep), not part of ms_owner */
    int64_t fwd_entries;     /* forward-list entries (= dyads) */
    int64_t map_items;       /* tag-map work items (pieces of <= 1024 dyads) */
    int64_t map_lookups;     /* lookup-list entries looked up in tag maps */
    int64_t map_triangles;   /* triangles found there */
    int64_t search_lookups;  /* lookup-list entries looked up by binary search */
    int64_t search_triangles;
    int64_t map_dyads;       /* dyad records of the tag-map owners */
    int64_t search_dyads;    /* dyad records of the other owners */
    int64_t map_list_entries;  /* forward-list entries of the tag-map items' owners */
    float ms_exact_cost;     /* TC_BIN_EXACT: the |S| pass before the task pass */
} tc_profile_t;

tc_status tc_census_profile(tc_profile_t* out);

/* tc_graph_build flags */
#define TC_DEVICE_PTRS 1u   /* src/dst (and arc offsets) are device pointers */
#define TC_UNDIRECTED 4u    /* each pair src[i], dst[i] is an undirected edge: both
                               arcs (a mutual dyad), the input mode of a Pajek
                               *Edges section (Sec. 5.1.1 reads both kinds) */
/* tc_census / tc_census_batched flags */
#define TC_OUT_DEVICE 2u    /* out is device memory: the call only enqueues work
                               on `stream` and returns without synchronising */

/* Fill *o with the defaults (tri_path TC_TRI_AUTO, fwd_big 64; for the merge
 * path degree-sum binning and tuned thresholds). */
tc_status tc_opts_default(tc_opts* o);

/*
 * tc_graph_build -- turn an arc list into the device adjacency the census reads
 * (the CRS "adjacency array" of Sec. 2.5.1 / 5.1.1, with the thesis's separate
 * edge and neighbour arrays folded into one list).
 *   n          vertex count, 0 <= n < 2^30.
 *   src, dst   m arc endpoints (arc src[i] -> dst[i]; with TC_UNDIRECTED
 *              the edge src[i] -- dst[i]), int32, host memory or, with
 *              TC_DEVICE_PTRS, device memory.  Not retained.
 *   m          number of arcs, >= 0.
 *   stream     stream the build runs on; the call synchronises it before
 *              returning (it reads back the graph statistics).
 *   out        receives the new graph handle.
 * Layout built on the device: row_ptr int64[n+1]; adj uint32[2|U|] where the
 * entry for neighbour y of row x is (y << 2) | tag, tag bit0 = arc x->y,
 * bit1 = arc y->x (3 = mutual dyad); each row sorted by neighbour id.
 * Errors: TC_ERR_ARG (null pointers with m > 0, n < 0, m < 0),
 * TC_ERR_UNSUPPORTED (n >= 2^30), TC_ERR_ID_RANGE, TC_ERR_OOM, TC_ERR_CUDA.
 */
tc_status tc_graph_build(int32_t n, const int32_t* src, const int32_t* dst, int64_t m,
                         uint32_t flags, void* stream, tc_graph* out);

/*
 * tc_graph_build_text -- a graph from a network file in the Pajek-style text
 * format the thesis reads (Sec. 4.2.1, "Implementation details": the order
 * of the graph, optional labelled vertex lines, then arcs of a directed or edges
 * of an undirected graph told apart by the section keyword; Sec. 5.1.1:
 * 0- or 1-based ids), parsed on the device, then built as tc_graph_build.
 *   text, bytes  the file's bytes (host memory or, with TC_DEVICE_PTRS,
 *                device memory; not retained), bytes < 2^31.
 *   id_base      0 or 1 (Pajek files are 1-based).
 * Lines: "*Vertices n" (required, once; its vertex lines are skipped),
 * "*Arcs" (lines "a b ...": arc a->b, further tokens such as weights are
 * ignored), "*Edges" ("a b ...": both arcs), "*Arcslist" / "*Edgeslist"
 * ("a b c ...": a->b, a->c, ... / edges); keywords case-insensitive; lines
 * starting with '%' and blank lines are skipped; '\r' counts as a blank.
 * Errors: TC_ERR_ARG (no or repeated *Vertices, data before any header, a
 * malformed header or arc line, bad id_base), TC_ERR_UNSUPPORTED (other
 * sections such as *Matrix, n >= 2^30, >= 2^30 arcs, text >= 2 GB),
 * TC_ERR_ID_RANGE (an id outside [base, base + n)), TC_ERR_OOM, TC_ERR_CUDA.
 */
tc_status tc_graph_build_text(const char* text, int64_t bytes, int32_t id_base, uint32_t flags, void* stream,
                              tc_graph* out);

/*
 * tc_graph_build_batched -- build G independent graphs in one pass.
 *   ns        host int32[G]: vertex count of each graph.
 *   arc_off   host int64[G+1]: graph g owns arcs arc_off[g] .. arc_off[g+1]-1
 *             of src/dst; arc_off[0] == 0.
 *   src, dst  concatenated arcs with ids LOCAL to their graph ([0, ns[g])).
 *   outs      receives G handles; they share one device allocation, which is
 *             released when the last of them is freed.
 * Errors as tc_graph_build; additionally sum(ns) must be < 2^31.
 */
tc_status tc_graph_build_batched(int32_t G, const int32_t* ns, const int64_t* arc_off,
                                 const int32_t* src, const int32_t* dst, uint32_t flags,
                                 void* stream, tc_graph* outs);

/* Statistics of one graph (host copy made at build time; no device work). */
tc_status tc_graph_stats(tc_graph g, tc_graph_stats_t* out);

/* Copy a graph's adjacency to host memory: row_ptr int64[n+1] (offsets
 * relative to the graph's first entry) and adj uint32[2*dyads] in the layout
 * described at tc_graph_build.  Synchronises the device. */
tc_status tc_graph_export(tc_graph g, int64_t* row_ptr, uint32_t* adj);

/*
 * tc_census -- the census of one graph (Sec. 2.2, Fig. "Subquadratic Triad
 * Census Algorithm"; task queues of Sec. 4.3.1 / 5.1.1).
 *   opts    NULL for the defaults.
 *   out     one tc_census_t, host memory (the call synchronises `stream`) or,
 *           with TC_OUT_DEVICE, device memory (asynchronous).
 * Errors: TC_ERR_ARG, TC_ERR_OOM (work space), TC_ERR_CUDA.
 */
tc_status tc_census(tc_graph g, const tc_opts* opts, tc_census_t* out, uint32_t flags,
                    void* stream);

/*
 * tc_census_batched -- censuses of G graphs in one pass over their combined
 * task set; out[i] is the census of gs[i].  All handles must come from ONE
 * tc_graph_build_batched (or be the same single graph); any subset and order
 * is allowed.  Errors as tc_census, plus TC_ERR_UNSUPPORTED for handles from
 * different builds.
 */
tc_status tc_census_batched(int32_t G, const tc_graph* gs, const tc_opts* opts,
                            tc_census_t* out, uint32_t flags, void* stream);

/*
 * Sharded census -- the census of G graphs of one build cut into `nshards`
 * shards whose accumulators add up, for callers that spread one census over
 * several processes or devices (the thesis names a multi-GPU system as
 * future work, Ch. 6).  Every canonical dyad's contributions are independent
 * (Sec. 2.2) and the only exchange is a sum: each shard runs the whole census
 * pipeline on the full graph (each process holds its own replica of the
 * build) but adds only its share, and the shares are summed word by word
 * (mod 2^64) before the fold and the 003 closure.
 *
 * tc_census_shard -- shard `shard` (0 <= shard < nshards) of the census of
 *   gs[0..G): the suffix and dyadic terms of the selection's adjacency
 *   entries [shard E / nshards, (shard+1) E / nshards) and the shared-
 *   neighbour corrections of the dyads owned by the rows [shard R / nshards,
 *   (shard+1) R / nshards) (E entries, R rows of the selection, graphs in
 *   the order given; with tri_path TC_TRI_AUTO, of each path's part).
 *   acc     device uint64[G][TC_ACC_WORDS]: graph i's raw accumulators (64
 *           codes, then sum (n - d_u - d_v) over the dyads with pre = 1, 2,
 *           3), overwritten.  Asynchronous on `stream`.
 * tc_census_fold -- out[i] (and/or codes[i]; either may be NULL) from the
 *   summed accumulators acc (device, [G][TC_ACC_WORDS]) of gs[i]: the 64->16
 *   fold, the common-neighbour share of the dyadic term and the 003 closure
 *   (k_fold).  out / codes are host memory (the call synchronises `stream`)
 *   or, with TC_OUT_DEVICE, device memory.
 * The sum over shards 0..nshards-1 of tc_census_shard's acc, folded, equals
 * tc_census_batched's result for the same graphs and opts.
 * Errors: TC_ERR_ARG, TC_ERR_UNSUPPORTED (handles from different builds),
 * TC_ERR_OOM, TC_ERR_CUDA.
 */
#define TC_ACC_WORDS 67
tc_status tc_census_shard(int32_t G, const tc_graph* gs, const tc_opts* opts, int32_t shard, int32_t nshards,
                          uint64_t* acc, void* stream);
tc_status tc_census_fold(int32_t G, const tc_graph* gs, const uint64_t* acc, tc_census_t* out,
                         tc_census64_t* codes, uint32_t flags, void* stream);

/*
 * tc_census_codes / tc_census_codes_batched -- the 64-code census of one
 * graph, or of G graphs of one build (out[i] for gs[i]); arguments, memory
 * and errors as tc_census / tc_census_batched.
 */
tc_status tc_census_codes(tc_graph g, const tc_opts* opts, tc_census64_t* out, uint32_t flags, void* stream);
tc_status tc_census_codes_batched(int32_t G, const tc_graph* gs, const tc_opts* opts, tc_census64_t* out,
                                  uint32_t flags, void* stream);

/*
 * tc_census_csr_noalloc -- the census of a graph the caller already holds in
 * device memory, computed WITHOUT ALLOCATING any device memory.  (The thesis
 * has no counterpart: this entry point exists for callers of this library.)
 *
 * Who needs it: callers that may not call cudaMalloc or any allocating
 * routine -- e.g. a host application whose memory manager owns the whole GPU
 * (a framework's caching allocator reserved it), a plugin that may only use
 * buffers handed to it, or a real-time service that forbids allocation after
 * start-up because an allocation can block and synchronise the device.
 *
 *   n        vertices, 0 <= n <= TC_NOALLOC_MAX_N.
 *   row_ptr  device int64[n+1], adj device uint32[nnz]: the tagged adjacency
 *            in exactly the layout tc_graph_build produces (see there; it can
 *            be copied out with tc_graph_export).  No padding is required.
 *   nnz      row_ptr[n] (= 2 * dyads), with nnz/2 <= TC_NOALLOC_MAX_DYADS.
 *   out      device tc_census_t, written by the call.
 *   stream   the work runs on it.  The call synchronises it twice (it reads
 *            back the CSR checks, then a capacity check), so it must never be
 *            made while `stream` is being captured into a CUDA graph: it then
 *            returns TC_ERR_ARG before enqueuing anything.
 * Scratch: a fixed area of about 5 MB compiled into the library as a static
 * device array; every GPU that loads the library holds it until the process
 * exits.  Each call looks up the array's device address on the current
 * device (cudaGetSymbolAddress, which allocates nothing; the first call on a
 * device loads the library's kernels there), so the address stays right
 * after the caller resets the device.  All calls share the one area and it
 * keeps the previous call's contents (the call clears what must start at
 * zero), so calls that overlap on the GPU -- from two streams or two host
 * threads -- race: serialise them.
 * Checks made on the device before any census kernel runs: row_ptr[0] == 0,
 * row_ptr[n] == nnz, no row offset decreases, every neighbour id < n.
 * Errors: TC_ERR_ARG (null pointers, negative or odd nnz, row offsets that
 * fail the checks, a capturing stream), TC_ERR_ID_RANGE (a neighbour id
 * outside [0, n)), TC_ERR_UNSUPPORTED (n or nnz/2 beyond the maxima, or the
 * CSR lists more canonical dyads than nnz/2, i.e. it is not symmetric; the
 * census is then not written correctly), TC_ERR_CUDA.
 */
#define TC_NOALLOC_MAX_N 262144
#define TC_NOALLOC_MAX_DYADS 262144
tc_status tc_census_csr_noalloc(int32_t n, const int64_t* row_ptr, const uint32_t* adj, int64_t nnz,
                                tc_census_t* out, void* stream);

/* MAN type index (0..15, order of tc_census_t) of the labelled triad with the
 * given 6-bit code, bit order of Sec. 2.2 Fig. "Triad Code Algorithm":
 * e(u,v)=1, e(v,u)=2, e(u,w)=4, e(w,u)=8, e(v,w)=16, e(w,v)=32 (the thesis's
 * TriadTable, whose printed form is lost).  Returns -1 for codes outside
 * [0, 64). */
int tc_triad_type(int code);

/*
 * Batch plans: the census of a fixed list of graphs recorded once as a CUDA
 * graph and replayed (the batched mode of the census; one persistent merge
 * launch when opts->persistent is set).
 *   tc_plan_create  gs: G >= 1 handles of ONE build (any subset/order);
 *                   opts: NULL = defaults, profile must be 0;
 *                   out: device tc_census_t[G], written by every run.
 *                   The plan owns its work space; creating it synchronises
 *                   `stream` and records the graph on a private stream.
 *   tc_plan_run     enqueue one replay on `stream` (asynchronous).
 *   tc_plan_free    synchronise the device and release the plan.
 * The graphs must outlive the plan.  Runs of one plan must not overlap.
 */
typedef struct tc_plan_s* tc_plan;
tc_status tc_plan_create(int32_t G, const tc_graph* gs, const tc_opts* opts, tc_census_t* out, void* stream,
                         tc_plan* plan);
tc_status tc_plan_run(tc_plan plan, void* stream);
void tc_plan_free(tc_plan plan);

/*
 * tc_autotune -- pick census options for a list of graphs by measurement:
 * coordinate descent over own_min, thr_thread, thr_warp, stream_max, chunk
 * and persistent (two passes), each trial a full census timed with CUDA events
 * on `stream` (best of two runs after a warm-up).  `base` (NULL = defaults)
 * is the starting point; max_trials <= 0 means no limit.  *best receives the
 * fastest options, *best_ms their time and *trials the number of options
 * timed.  The counts never depend on the options, only the time does.
 * Handles must come from one build, as for tc_census_batched.
 */
tc_status tc_autotune(int32_t G, const tc_graph* gs, const tc_opts* base, int32_t max_trials, void* stream,
                      tc_opts* best, float* best_ms, int32_t* trials);

/*
 * Learned cost model for task binning (opts.bin_mode = TC_BIN_MLP): an MLP
 * 8 -> 32 -> 32 -> 4 (ReLU) predicting log2 of the cycles a canonical-dyad
 * task takes in each bin (0 thread, 1 warp, 2 split tiles, 3 streamed).
 * The model decides the splitting of large tasks: every task above thr_warp
 * is streamed by one warp or cut into tiles, whichever it predicts cheaper
 * (k_route, FP16); smaller tasks keep the thr_thread / thr_warp rule.  The thesis bins by the degree sum |N(u)|+|N(v)|-2 (Sec. 4.3.1):
 * that rule remains the fallback while no model is installed.
 * Parameters: float[TC_MLP_NPARAM] = W1[32][8] b1[32] W2[32][32] b2[32]
 * W3[4][32] b3[4] (row = output neuron).  Features (float[8] per task,
 * shorter list s first): log2(1+d_s)/20, log2(1+d_g)/20, their difference,
 * log2(1+d_s+d_g)/20, mutual and out-only fractions of s and g.
 *
 *   tc_cost_sample      run the census with every eligible task forced into
 *                       `bin`, recording {u, v, bin, cycles} (int32 x 4, u/v
 *                       global rows) for tasks whose endpoint hash has
 *                       (hash & mask) == 0, at most `cap` records into the
 *                       device buffer `samples`; *n = records written.  Tiles
 *                       of a split task record one line each (same u, v).
 *   tc_cost_features    device features float[n][8] of tasks uv int32[n][2]
 *                       (global rows of the graph's build).
 *   tc_mlp_loss_grad    loss 1/n sum 0.5 (out[bin_i] - target_i)^2 and its
 *                       FP32 gradient float[TC_MLP_NPARAM] (device buffers).
 *   tc_mlp_train        `steps` Adam steps (lr, betas 0.9/0.999) on batches
 *                       of `batch` samples drawn with SplitMix64(seed); *loss
 *                       (device float) = loss over all n samples at the end.
 *   tc_mlp_predict      out float[n][4] from feat, in FP32 or, with
 *                       half_precision, the FP16 arithmetic binning uses.
 *   tc_cost_model_load  install host parameters on the current device for
 *                       TC_BIN_MLP (NULL uninstalls).
 */
#define TC_MLP_NPARAM 1476
tc_status tc_cost_sample(int32_t G, const tc_graph* gs, int32_t bin, int32_t mask, int32_t cap,
                         int32_t* samples, int32_t* n, void* stream);
tc_status tc_cost_features(tc_graph g, const int32_t* uv, int32_t n, float* feat, void* stream);
/* tc_union_sizes: |S| = |N(u) u N(v) \ {u, v}| (Sec. 2.2; the exact task
 * cost W3 of Sec. 4.3.1) of pairs uv int32[n][2] (device; global rows, both
 * of one graph of the build g belongs to) into out int32[n] (device);
 * synchronises `stream`.  Errors: TC_ERR_ARG, TC_ERR_ID_RANGE (a pair not
 * within one graph), TC_ERR_OOM, TC_ERR_CUDA. */
tc_status tc_union_sizes(tc_graph g, const int32_t* uv, int32_t n, int32_t* out, void* stream);
tc_status tc_mlp_loss_grad(const float* params, const float* feat, const int32_t* bin, const float* target,
                           int32_t n, float* grad, float* loss, void* stream);
tc_status tc_mlp_train(float* params, const float* feat, const int32_t* bin, const float* target, int32_t n,
                       int32_t steps, int32_t batch, float lr, uint64_t seed, float* loss, void* stream);
tc_status tc_mlp_predict(const float* params, const float* feat, int32_t n, int32_t half_precision, float* out,
                         void* stream);
tc_status tc_cost_model_load(const float* params);

/*
 * Path routing (tri_path = TC_TRI_AUTO).  The thesis has one way of finding
 * the shared neighbours; this library has two (forward lists, merge bins),
 * and which is faster depends on the graph: degree-skewed graphs (R-MAT,
 * power laws) favour the forward path, near-regular ones (G(n,p)) the merge
 * path.  A census of several graphs then runs each graph on its path.
 *   tc_path_features    float[G][8] (host) of G graphs: log2(1+n)/32,
 *                       log2(1+dyads)/32, log2(1+mean degree)/8,
 *                       log2(1+max degree)/20, log2(max/mean degree)/8,
 *                       log2(1+merged entries/dyads)/20, mutual fraction,
 *                       log2(1+merged entries)/40 (from the build statistics).
 *   tc_path_model_load  install host float[TC_MLP_NPARAM] (the 8-32-32-4 MLP
 *                       layout above; output 0 = predicted log2 census time of
 *                       a graph on the forward path, output 1 = on the merge
 *                       path) on the current device, evaluated in FP16; NULL
 *                       uninstalls.  Without a model the router uses the
 *                       degree-skew rule: the forward path when the largest
 *                       degree is at least 8x the mean degree.
 *   tc_path_route       path[i] (host int32[G]) = TC_TRI_FORWARD or
 *                       TC_TRI_MERGE for gs[i] (handles of one build).
 * The counts never depend on the route, only the time does.
 */
tc_status tc_path_features(int32_t G, const tc_graph* gs, float* feat);
tc_status tc_path_model_load(const float* params);
tc_status tc_path_route(int32_t G, const tc_graph* gs, int32_t* path, void* stream);

/* Release a graph handle (synchronises the device first). NULL is a no-op. */
void tc_graph_free(tc_graph g);

const char* tc_status_str(tc_status s);
const char* tc_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TC_H */
