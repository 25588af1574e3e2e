/*
 * hough.h -- C ABI of the GB300 conformal Hough hit filter (libhough.so).
 *
 * The library runs the hot path of the matrix-based conformal Hough transform
 * for drift-chamber hit filtering on an sm_103a GPU:
 *
 *   map     conformal map of every hit, Eq. (1) (with the factor 2 that makes
 *           Eq. (2) hold): u = 2x/r^2, v = 2y/r^2, in fixed point
 *           u_q = floor(2 x 2^32 / (x^2 + y^2)), x, y in integer micrometres
 *   rho     the hits x theta-bins matrix R of Sec. 3:
 *           rho_q(i, j) = u_q(i) c_j + v_q(i) s_j with c_j = round(2^14 cos th_j),
 *           s_j = round(2^14 sin th_j), th_j = (j + 1/2) pi / N_theta
 *   vote    k = clamp(floor((rho_q + H) N_rho / (2H)), 0, N_rho - 1), acc[j][k] += 1,
 *           H = 703687442 = 0.01 mm^-1 in units of 2^-46 um^-1 (the rho range
 *           [-0.01, 0.01] of Sec. 2); one int16 accumulator [N_theta][N_rho] per event
 *   peaks   cells with acc >= threshold that are 3x3 local maxima (Sec. 2 peak
 *           finding with neighbourhood suppression); ties: strictly above the
 *           neighbours that precede the cell in raster (theta-major) order, at least
 *           equal to those that follow; theta wraps (column -1 is column N_theta-1 and
 *           column N_theta is column 0, both with k -> N_rho-1-k); neighbours past the
 *           rho edges are skipped; peaks listed in raster order
 *   select  back-projection filter (Sec. 2 "data filtering"): a hit is kept when, at
 *           the theta column of some stored peak, its rho bin is within
 *           keep_halfwidth of the peak's rho bin
 *
 * All arithmetic is integer, so results are exact and reproducible.
 *
 * Conventions for every entry point:
 *   - Pointers named d_* are DEVICE pointers owned by the caller; h_* are host
 *     pointers. The library allocates no device memory in any entry point.
 *   - Hits: int32 (x, y) pairs in micrometres, |x|, |y| <= 2^24, stored
 *     interleaved (8 bytes per hit, 8-byte aligned). Event e owns hits
 *     [off[e], off[e+1]) of an int64 offsets array with off[0] = 0,
 *     non-decreasing, off[n_events] = n_hits.
 *   - Work is enqueued asynchronously on `stream` (a cudaStream_t passed as void*,
 *     NULL = legacy default stream) and the call returns without synchronising.
 *   - Return value: HOUGH_OK or a negative HOUGH_E* code for faults the host can
 *     see (nothing is enqueued then). Faults only the device can see are OR-ed as
 *     HOUGH_F_* bits into the caller's status buffer d_status (int32[4], zeroed by
 *     the caller before first use; word 0 holds the sticky flags, words 1..3 are
 *     per-call scratch). Read it with hough_status(). Calls that run concurrently
 *     must use distinct status buffers.
 *   - A hit with r = 0 or a coordinate beyond 2^24 um sets HOUGH_F_BAD_HIT and
 *     neither votes nor is kept. An event with more than HOUGH_MAX_EVENT_HITS
 *     hits sets HOUGH_F_EVENT_TOO_LARGE and yields zero accumulator, no peaks and
 *     no kept hits. Offsets that break the rules above set HOUGH_F_BAD_OFFSETS
 *     and no output of that call is written.
 */
#ifndef HOUGH_H
#define HOUGH_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define HOUGH_OK 0
#define HOUGH_EINVAL (-1)     /* null pointer or negative count */
#define HOUGH_EPARAM (-2)     /* hough_params out of range */
#define HOUGH_ESMEM (-3)      /* requested shape does not fit shared memory */
#define HOUGH_ECUDA (-4)      /* CUDA runtime error (see hough_last_cuda_error) */
#define HOUGH_EWORKSPACE (-5) /* workspace too small */
#define HOUGH_ETIMEDOUT (-6)  /* a bounded wait gave up */
#define HOUGH_EFULL (-7)      /* serving admission refused: no free slot */
#define HOUGH_EDEVICE (-8)    /* device-side status flags are set */

/* ---- device status flags (word 0 of d_status) ---- */
#define HOUGH_F_BAD_HIT 1
#define HOUGH_F_BAD_OFFSETS 2
#define HOUGH_F_PEAK_OVERFLOW 4 /* an event had more than max_peaks peaks: the first
                                   max_peaks in raster order are stored and used */
#define HOUGH_F_EVENT_TOO_LARGE 8
#define HOUGH_F_TIMEOUT 16       /* serving: the request's micro-batch did not complete within
                                    HOUGH_SERVE_BATCH_TIMEOUT_NS; its outputs were not written */
#define HOUGH_F_LAUNCH_FAILED 32 /* serving: the request's micro-batch could not be enqueued (a
                                    CUDA error); its outputs were not written */

#define HOUGH_STATUS_WORDS 4
#define HOUGH_MAX_EVENT_HITS 32767
#define HOUGH_RHO_HALF_RANGE 703687442LL /* H */

/* Algorithm and launch parameters. Zero in a launch field means "choose". */
typedef struct hough_params {
  int32_t n_theta;        /* N_theta in [4, 1024] */
  int32_t n_rho;          /* N_rho in [4, 1024] */
  int32_t threshold;      /* absolute vote threshold, >= 1 */
  int32_t keep_halfwidth; /* rho-bin half-width of the selection window, >= 0 */
  int32_t max_peaks;      /* stored peaks per event, in [1, 65536] */
  int32_t theta_tiles;    /* theta tiles per event (0 = auto); each tile is one CTA */
  int32_t events_per_cta; /* persistent queue: work items taken per pop (0 = auto) */
  int32_t block;          /* threads per CTA (0 = auto) */
  /* Peak finder (Sec. 2). HOUGH_PEAK_LOCAL_MAX (0, the default): one pass of 3x3 local maxima
   * >= threshold, listed in raster order. HOUGH_PEAK_ITERATIVE (1): the paper's own finder. A
   * cell qualifies iff acc >= threshold and acc * rel_den >= rel_num * max(acc) (a fraction of
   * the accumulator's maximum, exact in integers). The qualifying cell with the most votes
   * that is not yet suppressed (ties: the first in raster order) becomes the next peak, and
   * every cell within nms_radius of it in theta and rho is suppressed. Theta wraps with rho
   * mirrored, and rows beyond the rho edges are skipped. Peaks are listed in extraction order.
   * The iterative finder needs the whole accumulator in one CTA on the fused paths
   * (theta_tiles 1); the stepwise hough_peaks takes any size. */
  int32_t peak_mode;
  int32_t rel_num;        /* mode 1: numerator of the relative threshold, 0 <= rel_num <= rel_den */
  int32_t rel_den;        /* mode 1: denominator, >= 1 */
  int32_t nms_radius;     /* mode 1: suppression half-width in bins, 0 <= 2 nms_radius < n_theta, <= 64 */
} hough_params;

#define HOUGH_PEAK_LOCAL_MAX 0
#define HOUGH_PEAK_ITERATIVE 1

/* One peak: theta bin j, rho bin k, votes acc[j][k], flags (reserved, 0). 8 bytes. */
typedef struct hough_peak {
  int16_t theta_bin;
  int16_t rho_bin;
  int16_t votes;
  int16_t flags;
} hough_peak;

/* ---- stepwise entry points (the accumulator goes through HBM; used for parity) ---- */

/* Conformal map, Eq. (1)/(2): d_uq[i], d_vq[i] = u_q, v_q of hit i (int64, n_hits each).
 * A bad hit gets INT64_MIN in both and sets HOUGH_F_BAD_HIT. d_off is validated only. */
int hough_map(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events, int64_t* d_uq,
              int64_t* d_vq, int32_t* d_status, void* stream);

/* Voting over the rho matrix (Sec. 3): d_acc = int16 [n_events][n_theta][n_rho], raster
 * (theta-major) order, fully overwritten. Hits whose d_uq is INT64_MIN are skipped. */
int hough_vote(const int64_t* d_uq, const int64_t* d_vq, int64_t n_hits, const int64_t* d_off, int64_t n_events,
               const hough_params* p, int16_t* d_acc, int32_t* d_status, void* stream);

/* Peak finding with neighbourhood suppression (Sec. 2, peak finding; the peak_mode field of
 * hough_params selects the 3x3 local-maximum reading or the paper's iterative finder) on d_acc
 * (layout as written by hough_vote): d_npeaks[e] = true peak count,
 * d_peaks = [n_events][max_peaks], the first min(count, max_peaks) in raster order; entries past
 * them are left unchanged (this holds for every entry point that writes peaks). */
int hough_peaks(const int16_t* d_acc, int64_t n_events, const hough_params* p, int32_t* d_npeaks,
                hough_peak* d_peaks, int32_t* d_status, void* stream);

/* Back-projection selection (Sec. 2, data filtering: the hits lying on a found peak's curve are
 * kept): d_mask[i] = 1 if hit i is kept, else 0; d_nkept[e] = kept hits of e. */
int hough_select(const int64_t* d_uq, const int64_t* d_vq, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                 const hough_params* p, const int32_t* d_npeaks, const hough_peak* d_peaks, uint8_t* d_mask,
                 int32_t* d_nkept, int32_t* d_status, void* stream);

/* Circle recovery, Eq. (2): for each stored peak (theta_bin j, rho_bin k) of each event, the
 * circle through the origin it stands for, at the bin centres th = (j + 1/2) pi / n_theta and
 * rho = (-1 + (2k + 1) / n_rho) * 0.01 mm^-1 (Sec. 2): d_circles[(e * max_peaks + q) * 4 + 0..3]
 * = x_c = cos(th) / rho, y_c = sin(th) / rho (mm), r_c = 1 / |rho| (mm) and
 * pT = 0.3 * b_tesla * r_c (MeV/c), as float (computed in double). Only the first
 * min(d_npeaks[e], max_peaks) records of each event are read and written; the rest of
 * d_circles is left unchanged. A rho bin centre of 0 (odd n_rho) gives infinite radius. Uses
 * n_theta, n_rho and max_peaks of p. Enqueued on `stream`; HOUGH_EINVAL for null pointers. */
int hough_circles(const int32_t* d_npeaks, const hough_peak* d_peaks, int64_t n_events, const hough_params* p,
                  double b_tesla, float* d_circles, void* stream);

/* ---- fused path (the accumulator never leaves shared memory) ---- */

/* Device workspace bytes that hough_run / hough_run_batched need for these parameters
 * and batch size (0 is never returned). */
size_t hough_workspace_size(const hough_params* p, int64_t n_events);

/* Whole path in one pass: map -> rho -> vote -> peaks -> select for every event (Eq. 1, the
 * matrix R of Sec. 3, Sec. 2 peak finding and data filtering), one CTA per event or theta tile:
 * the event-level parallelism of Sec. 3.
 * Outputs as in the stepwise calls; d_checksum (nullable) gets per event
 * sum over cells c = j*n_rho + k of acc[c] * splitmix64_finalizer(c + 1) mod 2^64.
 * d_ws: workspace of ws_bytes >= hough_workspace_size(p, n_events), 256-byte aligned.
 * d_xy and d_peaks must be 8-byte aligned (each record is written as one 8-byte store);
 * otherwise HOUGH_EINVAL. One CTA per (event, theta tile). */
int hough_run(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events, const hough_params* p,
              int32_t* d_npeaks, hough_peak* d_peaks, uint8_t* d_mask, int32_t* d_nkept, uint64_t* d_checksum,
              void* d_ws, size_t ws_bytes, int32_t* d_status, void* stream);

/* Same results as hough_run, scheduled as one persistent launch over the batch (Sec. 3, events
 * processed in parallel as a batch; Sec. 4 measures batches of events): CTAs pop
 * (event, tile) work items, largest events first, from a queue in d_ws. The
 * validation/ordering kernel and the persistent kernel are replayed as a CUDA
 * graph cached per (pointers, sizes, parameters, stream). */
int hough_run_batched(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                      const hough_params* p, int32_t* d_npeaks, hough_peak* d_peaks, uint8_t* d_mask,
                      int32_t* d_nkept, uint64_t* d_checksum, void* d_ws, size_t ws_bytes, int32_t* d_status,
                      void* stream);

/* End-to-end form for callers holding HOST buffers (pinned memory recommended): copies
 * h_xy/h_off to the device, runs the batched path, packs the stored peaks densely and
 * copies the results back, then synchronises `stream`. Outputs: h_npeaks[n_events] (true
 * counts), h_peak_off[n_events + 1] (offsets of each event's stored peaks in h_peaks),
 * h_peaks[<= h_peaks_cap], h_mask[n_hits], h_nkept[n_events]. d_buf is a device staging
 * buffer of d_buf_bytes >= hough_host_buffer_size(p, n_hits, n_events) bytes, 256-byte
 * aligned. Returns HOUGH_EWORKSPACE if the stored peaks exceed h_peaks_cap (h_peak_off is
 * valid then), or HOUGH_EDEVICE if device flags were raised (outputs are valid). */
int hough_run_host(const int32_t* h_xy, int64_t n_hits, const int64_t* h_off, int64_t n_events, const hough_params* p,
                   int32_t* h_npeaks, int64_t* h_peak_off, hough_peak* h_peaks, int64_t h_peaks_cap, uint8_t* h_mask,
                   int32_t* h_nkept, void* d_buf, size_t d_buf_bytes, int32_t* d_status, void* stream);

/* Device staging bytes hough_run_host needs. */
size_t hough_host_buffer_size(const hough_params* p, int64_t n_hits, int64_t n_events);

/* Stages of hough_run_host, the analogue of the paper's per-stage study (Sec. 4: transfers,
 * voting, peak finding, result transfer), for hough_host_stage_ms: busy milliseconds of each
 * stage summed over the call's event chunks (the chunks' stages overlap one another), and the
 * span from the call's first enqueued work to its last copy. */
#define HOUGH_HOST_STAGE_H2D 0       /* hits and offsets to the device (and offset rebasing) */
#define HOUGH_HOST_STAGE_KERNELS 1   /* validation + fused kernel: map, vote, peaks, select */
#define HOUGH_HOST_STAGE_PACK 2      /* stored peaks packed densely */
#define HOUGH_HOST_STAGE_D2H 3       /* counts, kept masks and peak offsets to the host */
#define HOUGH_HOST_STAGE_PEAKS_D2H 4 /* packed peaks to the host */
#define HOUGH_HOST_STAGE_SPAN 5      /* first work to last copy, on the device clock */
#define HOUGH_HOST_STAGES 6

/* Measurement hook for the calling host thread: with on != 0, later hough_run_host calls
 * record CUDA timing events around every stage of every chunk (on the stage's own stream). */
void hough_set_host_timing(int32_t on);

/* Stage times of this thread's last timed hough_run_host call: min(n, HOUGH_HOST_STAGES)
 * values in ms into ms. HOUGH_EINVAL if that call was not timed or did not complete. */
int hough_host_stage_ms(float* ms, int32_t n);

/* Measurement hook for the calling host thread: when both are non-NULL, later fused and
 * batched calls record the CUDA events begin/end (cudaEvent_t passed as void*) on their
 * stream immediately before and after the main fused kernel, so its duration can be read
 * with cudaEventElapsedTime. NULL, NULL turns it off. Graph replays are cached per pair. */
void hough_set_stage_events(void* begin, void* end);

/* ---- serving loop (continuous batching) ---- */

/* Configuration of a serving loop. Requests (one event each) are admitted into micro-batches;
 * up to `slots` micro-batches are in flight at once, each on its own stream with its own
 * device and pinned host buffers, so new arrivals are gathered while earlier ones run. A
 * micro-batch is launched when it holds max_batch_events events or max_batch_hits hits, or
 * when its oldest request has waited flush_ns (0: only when full, or on drain). */
typedef struct hough_serve_config {
  hough_params params;
  int32_t slots;            /* micro-batches in flight, 1..64 */
  int32_t max_batch_events; /* events per micro-batch, >= 1 */
  int64_t max_batch_hits;   /* hits per micro-batch, >= 1 (also the largest admissible event) */
  int64_t flush_ns;         /* longest wait of a request before its partial batch is launched */
  int32_t queue_capacity;   /* requests waiting for a slot before submit refuses (HOUGH_EFULL); the
                               ring of results not yet polled holds queue_capacity plus the
                               in-flight requests, and a request is admitted only with room there */
  int32_t reserved;
} hough_serve_config;

/* Longest wait of the serving loop for one micro-batch; past it the batch's requests finish
 * with HOUGH_F_TIMEOUT and its slot is retired (never reused). */
#define HOUGH_SERVE_BATCH_TIMEOUT_NS 10000000000LL

/* One finished request. Latency = t_done_ns - t_arrival_ns (steady clock, ns): from the
 * request's arrival (its submit call, or its scheduled time in hough_serve_replay) to the
 * moment its results were in host memory. A request whose status has HOUGH_F_TIMEOUT or
 * HOUGH_F_LAUNCH_FAILED set has no results: npeaks and nkept are 0 and its output buffers
 * were not written. */
typedef struct hough_serve_result {
  int64_t id;
  int32_t status; /* HOUGH_F_* flags raised by the micro-batch the request ran in */
  int32_t npeaks; /* true peak count */
  int32_t nkept;  /* kept hits */
  int32_t reserved;
  int64_t t_arrival_ns;
  int64_t t_done_ns;
} hough_serve_result;

/* Device and pinned-host bytes a server with this configuration needs. */
int hough_serve_buffer_sizes(const hough_serve_config* c, size_t* device_bytes, size_t* pinned_bytes);

/* Starts a server on the current device. d_buf (device) and h_pinned (page-locked host
 * memory) are caller-owned, 256-byte aligned and must outlive the server. *server receives
 * an opaque handle. A host thread owned by the server runs the loop until hough_serve_close.
 * The server's own host memory (request queue, results ring, per-slot lists) is allocated and
 * written here, once: the serving path neither allocates nor touches fresh pages. */
int hough_serve_open(const hough_serve_config* c, void* d_buf, size_t d_bytes, void* h_pinned, size_t h_bytes,
                     void** server);

/* Admits one event (h_xy: n_hits interleaved int32 (x, y) pairs, read when its micro-batch is
 * gathered, so it must stay valid until the request completes). On completion its kept mask
 * (n_hits bytes) and stored peaks (up to max_peaks records) are copied to h_mask_out /
 * h_peaks_out when non-NULL. Returns HOUGH_EFULL when queue_capacity requests are waiting. */
int hough_serve_submit(void* server, const int32_t* h_xy, int64_t n_hits, int64_t id, uint8_t* h_mask_out,
                       hough_peak* h_peaks_out);

/* Moves up to max_results finished requests into out; *n_out gets the count. */
int hough_serve_poll(void* server, hough_serve_result* out, int32_t max_results, int32_t* n_out);

/* Launches any partial micro-batch and waits until every admitted request has finished, or
 * timeout_ns elapsed (HOUGH_ETIMEDOUT). */
int hough_serve_drain(void* server, int64_t timeout_ns);

/* Replays an arrival schedule from the calling thread: request i (id i) is event
 * (i mod pool_events) of the pool (h_off_pool offsets into h_xy_pool) and is submitted at
 * t0 + arrival_ns[i] (busy wait), t0 written to *t_start_ns. A refused admission is retried
 * for up to 10 s with the same scheduled arrival time. Results are copied out when the
 * buffers are given (each nullable): request i's kept mask to h_mask_out + m_i, where m_i is
 * the sum of the hit counts of requests 0 .. i-1, its stored peaks to h_peaks_out + i * max_peaks,
 * and its result record to h_results_out[i] (then it does not go to the results ring and
 * hough_serve_poll does not return it; write the array once beforehand, so that the loop does
 * not fault its pages in). */
int hough_serve_replay(void* server, const int32_t* h_xy_pool, const int64_t* h_off_pool, int64_t pool_events,
                       const int64_t* arrival_ns, int64_t n_requests, int64_t* t_start_ns, uint8_t* h_mask_out,
                       hough_peak* h_peaks_out, hough_serve_result* h_results_out);

/* Stops the loop, waits for the streams and releases the handle. */
int hough_serve_close(void* server);

/* Timing record of one micro-batch (steady clock, ns), kept by the serving loop in a ring of
 * the HOUGH_SERVE_RECORDS most recent batches. */
typedef struct hough_serve_batch_record {
  int64_t t_gather;    /* the loop took the batch's requests from the queue */
  int64_t t_launched;  /* its copies and kernels were enqueued */
  int64_t t_done_seen; /* the loop saw its completion event */
  int64_t t_finished;  /* its results were in the callers' buffers and queued */
  int64_t n_hits;
  int32_t n_events;
  int32_t slot;
} hough_serve_batch_record;

#define HOUGH_SERVE_RECORDS 65536

/* Stalls of one thread: gaps of more than stall_ns between its consecutive ticks (passes of the
 * serving loop, or iterations of hough_serve_replay's submitter, which ticks while it waits for
 * the next scheduled arrival). For the longest gap, the thread's usage over its window (the gap
 * plus at most 1 ms before it, sampled with getrusage): CPU time near the window means it was
 * busy (system time and minor faults: in the kernel, e.g. faulting pages in); near zero that it
 * was not running (voluntary switches: blocked; involuntary ones: preempted). */
typedef struct hough_serve_stall {
  int64_t count;
  int64_t max_gap_ns;
  int64_t max_gap_at; /* when the longest gap began (steady clock, ns) */
  int64_t user_ns, sys_ns;
  int64_t minor_faults;
  int64_t voluntary_switches, involuntary_switches;
} hough_serve_stall;

/* Health of the serving loop and of hough_serve_replay's submitter, for finding stalls. */
typedef struct hough_serve_stats {
  int64_t passes;           /* passes of the serving loop */
  int64_t batches;          /* micro-batches launched */
  int64_t stall_ns;         /* threshold (1 ms) */
  hough_serve_stall loop;   /* the serving loop's thread */
  hough_serve_stall submit; /* the thread of the last hough_serve_replay */
} hough_serve_stats;

/* Copies the loop's statistics into *out, and up to max_records of the most recent batch
 * records (oldest first) into records (nullable); *n_records (nullable) gets their count. */
int hough_serve_trace(void* server, hough_serve_stats* out, hough_serve_batch_record* records, int32_t max_records,
                      int32_t* n_records);

/* Test hook: the next n micro-batch launches of this server fail on the host before anything
 * is enqueued, as a CUDA launch error would; their requests finish with HOUGH_F_LAUNCH_FAILED. */
int hough_serve_inject_launch_failures(void* server, int32_t n);

/* Size of the library's built-in scratch array used by hough_run_batched_static. */
#define HOUGH_STATIC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* hough_run_batched for callers that cannot allocate device memory (the paper has no
 * counterpart; it is an interface convenience). Examples: a plain-C trigger process whose
 * only device buffers are the input and output buffers its readout layer mapped once, or a
 * real-time loop that must not call cudaMalloc after start-up because an allocation can
 * synchronise the device. The caller passes inputs and outputs exactly as for
 * hough_run_batched but no workspace: the scratch (queue counter, event order, tile peak
 * slots) comes from a HOUGH_STATIC_SCRATCH_BYTES array compiled into the library, which
 * every GPU that loads the library keeps until the process exits. Batches whose scratch,
 * hough_workspace_size(p, n_events), exceeds that size are rejected with HOUGH_EWORKSPACE.
 * The call allocates nothing. The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress, with that device current), so make that first call before
 * any stream capture. That address is kept for the life of the process: after cudaDeviceReset on
 * a device, do not call this entry point on that device again. All calls share the one array: calls that can overlap on the GPU (on
 * different streams or host threads) race and must be serialised by the caller. Results are
 * identical to hough_run_batched (the same kernels run, launched directly, without a graph). */
int hough_run_batched_static(const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                             const hough_params* p, int32_t* d_npeaks, hough_peak* d_peaks, uint8_t* d_mask,
                             int32_t* d_nkept, uint64_t* d_checksum, int32_t* d_status, void* stream);

/* Autotuner of the batched path: times hough_run_batched's kernels on the sample batch
 * (d_xy, d_off: device, the caller's representative events) for every feasible launch shape
 * -- theta tiles in {1, 2, 4, 8, 16}, threads per CTA in {256, 512, 1024} (or the widest the
 * tiling allows), queue items per pop (events_per_cta) in {1, 2, 4} -- and writes the fastest
 * into *p (theta_tiles, block, events_per_cta; the algorithm fields are untouched). d_scratch
 * holds outputs and workspace of every candidate: hough_autotune_scratch_size bytes, 256-byte
 * aligned. Results are cached per (parameters, device, SM count, hits per event in octaves);
 * a cached answer returns at once with *best_ms = -1. Synchronises `stream`. */
size_t hough_autotune_scratch_size(const hough_params* p, int64_t n_hits, int64_t n_events);
int hough_autotune(hough_params* p, const int32_t* d_xy, int64_t n_hits, const int64_t* d_off, int64_t n_events,
                   void* d_scratch, size_t scratch_bytes, int32_t* d_status, void* stream, float* best_ms);

/* Launch shape the library would use for these parameters: fills the zero launch fields
 * of *p (theta_tiles, events_per_cta, block) and returns HOUGH_OK or an error. */
int hough_resolve_params(hough_params* p);

/* Synchronises `stream`, copies word 0 of d_status into *host_flags and returns
 * HOUGH_OK if it is 0, else HOUGH_EDEVICE. */
int hough_status(const int32_t* d_status, void* stream, int32_t* host_flags);

/* Static description of a return code or of a single HOUGH_F_* flag value. */
const char* hough_strerror(int code);

/* Last CUDA runtime error code seen by the library on this host thread (0 if none). */
int hough_last_cuda_error(void);

/* ---- measurement and self-test entry points ---- */

/* Exhaustively checks the device rho-bin function against plain 64-bit integer
 * division over rho in [rho_lo, rho_hi]: *d_mismatch (uint64, caller-zeroed) gets
 * the number of disagreements. */
int hough_selftest_bin(int32_t n_rho, int64_t rho_lo, int64_t rho_hi, unsigned long long* d_mismatch,
                       void* stream);

/* Checks the vote's float bin paths (a float estimate of the bin, exact integer arithmetic
 * whenever an integer lies within the estimate's error bound of it) on n_samples
 * pseudo-random (u_q, v_q, column) tuples of the int32 fast-path range against plain 64-bit
 * floor division. d_out[5] (uint64, caller-zeroed): [0] disagreements of the general
 * estimate, [1] its tuples that took the exact integer path, [2] disagreements of the
 * mirror-pair layout's bit-pattern row (tuples with u^2 + v^2 inside its fast-path disc),
 * [3] those that took its exact path, [4] the tuples inside the disc. */
int hough_selftest_fpbin(int32_t n_theta, int32_t n_rho, uint64_t seed, int64_t n_samples, unsigned long long* d_out,
                         void* stream);

/* Shared-memory atomic ceiling: every SM runs `ctas_per_sm` CTAs of `threads` threads,
 * each thread issuing `iters` x 16 32-bit shared-memory adds into a `smem_bytes`
 * array with address pattern `mode` (0: each lane its own bank, conflict-free;
 * 1: pseudo-random words; 2: all lanes of a warp on one word; 3: each thread always on
 * the same word of its own bank, so consecutive adds of a thread hit one address; 4: each lane
 * on its own bank at pseudo-random rows, the access pattern of the mirror-pair vote).
 * *d_sink receives a
 * value that keeps the work alive. Time it with events on `stream`. */
int hough_probe_smem_atomics(int32_t mode, int32_t ctas_per_sm, int32_t threads, int32_t smem_bytes, int32_t iters,
                             unsigned long long* d_sink, void* stream);

/* Phases of a fused-kernel item, in order, for hough_phase_cycles. The iterative finder's
 * phases replace the scan's; SCAN is then the accumulator checksum before the finder. */
#define HOUGH_PHASE_CLEAR 0         /* zero the accumulator, halo and peak bitmap */
#define HOUGH_PHASE_STAGE 1         /* map hits into shared memory (all chunks) */
#define HOUGH_PHASE_VOTE 2          /* votes (all chunks) */
#define HOUGH_PHASE_FOLD 3          /* guard rows of the mirror-pair layout */
#define HOUGH_PHASE_SCAN 4          /* 3x3 local-maximum scan (or the checksum, iterative finder) */
#define HOUGH_PHASE_EXSCAN 5        /* block scan of the peak-record keys */
#define HOUGH_PHASE_RECORDS 6       /* peak records */
#define HOUGH_PHASE_MERGE 7         /* theta tiles: publish and merge */
#define HOUGH_PHASE_IT_MAX 8        /* iterative finder: accumulator maximum */
#define HOUGH_PHASE_IT_COLLECT 9    /* iterative finder: candidates */
#define HOUGH_PHASE_IT_RESOLVE 10   /* iterative finder: kept set (rounds, walk or passes) */
#define HOUGH_PHASE_IT_ORDER 11     /* iterative finder: kept keys sorted, records */
#define HOUGH_PHASE_SEL_COLUMNS 12  /* selection: peak columns and their trig values */
#define HOUGH_PHASE_SEL_BITMAPS 13  /* selection: dilated peak bitmaps */
#define HOUGH_PHASE_SEL_A 14        /* selection: a lane per hit over the first peak columns */
#define HOUGH_PHASE_SEL_B 15        /* selection: the rest, and the event outputs */
#define HOUGH_PHASE_COUNT 16

/* Per-phase cycle counters of the fused kernel, in a library built with HOUGH_PHASE_TIMERS
 * defined (`_build.build(variant="phase")`): thread 0 of every CTA adds the clock64() cycles
 * since its previous mark to the counter of the phase that just ended, so a counter over a
 * launch divided by its events is the cycles an event spends in that phase on one SM.
 * Synchronises the device, copies min(n, HOUGH_PHASE_COUNT) counters to host_cycles and,
 * with reset != 0, zeroes them. *enabled (may be null) is 1 in the timer build and 0
 * otherwise (the counters then read 0). HOUGH_EINVAL for a null host_cycles or n < 0. */
int hough_phase_cycles(uint64_t* host_cycles, int32_t n, int32_t reset, int32_t* enabled);

#ifdef __cplusplus
}
#endif

#endif /* HOUGH_H */
