/*
 * ntbc.h -- C ABI of the GB300 (sm_103a) implementation of Neural Texture Block
 * Compression (Fujieda & Harada, "Neural Texture Block Compression", 2024).
 *
 * Conventions shared by every entry point
 *   - Every call returns an ntbc_status; NTBC_OK is 0. On failure the calling
 *     thread's message is available from ntbc_last_error(). Nothing throws,
 *     aborts or traps.
 *   - Arguments are validated on the host before any launch; invalid shapes or
 *     pointers give NTBC_EINVAL and launch nothing.
 *   - Data pointers are DEVICE pointers owned by the caller unless the comment
 *     says "host". `stream` is a cudaStream_t (NULL = legacy default stream);
 *     calls are asynchronous on it unless the comment says otherwise.
 *   - Textures are row-major uint8: RGB8 (3 bytes per texel) for BC1, R8 for BC4,
 *     pitch = width * channels. Width and height are positive multiples of 4.
 *   - Compressed textures are (width/4)*(height/4) blocks of 8 bytes in
 *     row-major block order (Sec. 1: "BC1 and BC4 compress each block to 8 bytes").
 *     Within a block texel i = 4*y + x. BC1: bytes 0-1 colour0, 2-3 colour1
 *     (little-endian RGB565, R in bits 15..11), bytes 4-7 little-endian u32 with
 *     texel i's 2-bit code in bits 2i..2i+1. BC4: byte 0 r0, byte 1 r1, bytes 2-7
 *     little-endian 48-bit field with texel i's 3-bit code in bits 3i..3i+2.
 */
#ifndef NTBC_H
#define NTBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NTBC_OK = 0,
    NTBC_EINVAL = 1,        /* bad argument; nothing was launched */
    NTBC_ENOMEM = 2,        /* device allocation failed */
    NTBC_ECUDA = 3,         /* a CUDA runtime call or launch failed */
    NTBC_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
    NTBC_ENONFINITE = 5,    /* training produced a non-finite loss */
    NTBC_EUNSUPPORTED = 6   /* valid request outside what the kernels implement */
} ntbc_status;

enum { NTBC_BC1 = 1, NTBC_BC4 = 4 };
/*
 * Compositions of the two (Sec. 2.1: BC2, BC3 and BC5 combine BC1 and BC4), 16-byte blocks,
 * accepted by the codec (bc_reference_encode, bc_decode):
 *   NTBC_BC3  RGBA8 texels; bytes 0-7 the alpha channel as a BC4 block, bytes 8-15 the colour
 *             as a BC1 block that always decodes with the four-colour palette
 *   NTBC_BC5  two-channel texels (2 bytes each); bytes 0-7 channel 0 as a BC4 block, bytes
 *             8-15 channel 1
 * A model encodes them as their parts (a BC1 and a BC4 texture, or two BC4 textures) and
 * writes the interleaved blocks with ntbc_infer_to_bc_strided.
 */
enum { NTBC_BC3 = 3, NTBC_BC5 = 5 };
enum { NTBC_ACT_SELU = 0, NTBC_ACT_RELU = 1 };
/*
 * Inference precision (the stored MLP weights are FP16 for the two FP16 modes):
 *   NTBC_PREC_FP32       FP32 weights and arithmetic (SIMT kernel)
 *   NTBC_PREC_FP16       FP16 weights on tensor cores (tcgen05, FP32 accumulation); each
 *                        activation enters the MMA as an FP16 pair hi + lo (two passes), so
 *                        the outputs stay within 1e-3 relative of an FP64 evaluation
 *   NTBC_PREC_FP16_FAST  FP16 weights and FP16 activations (one pass), the paper's half-
 *                        precision inference (Sec. 3.3); outputs within about 4e-3 relative
 *   NTBC_PREC_FP8        MLP weights and biases stored as FP8 E4M3 codes (round to nearest
 *                        even, saturating at +-448) with one power-of-two scale 2^e per
 *                        layer, e the smallest integer with max|w| <= 448 * 2^e; the values
 *                        q * 2^e are exact in FP16 and run on the NTBC_PREC_FP16 path (split
 *                        activations), so the outputs stay within 1e-3 relative of an FP64
 *                        evaluation with the same FP8 weights. The paper stores FP16 weights;
 *                        this mode is an extension for the weight-precision study (FP8
 *                        storage, FP16 arithmetic).
 *   NTBC_PREC_FP8_MMA    FP8 arithmetic: the NTBC_PREC_FP8 weights, and every layer's input
 *                        (grid features, hidden activations) rounded to E4M3 (nearest even,
 *                        saturating) at a per-layer power-of-two scale 2^a; the MMAs are
 *                        tcgen05 kind::f8f6f4 (E4M3 x E4M3, FP32 accumulation in TMEM), the
 *                        biases (the FP8 values) are added in FP32 after the MMA. a is the
 *                        smallest integer with 2 max|x| <= 448 * 2^a over a calibration sample
 *                        taken at export: 2048 blocks (all, if fewer) at ids
 *                        i * 2654435761 mod n_blocks, the endpoint network on their centres
 *                        and the colour network on their 16 texels, evaluated in FP32 with the
 *                        FP8 weights and unrounded activations. Outputs match an FP64
 *                        evaluation of the same arithmetic except where an FP32 activation
 *                        lands on the other side of an E4M3 rounding boundary; against exact
 *                        activations they differ by a few per cent. An extension for the
 *                        precision study, like NTBC_PREC_FP8.
 */
enum { NTBC_PREC_FP32 = 0, NTBC_PREC_FP16 = 1, NTBC_PREC_FP16_FAST = 2, NTBC_PREC_FP8 = 3, NTBC_PREC_FP8_MMA = 4 };

#define NTBC_MAX_TEXTURES 8
#define NTBC_MAX_LEVELS 16
#define NTBC_MAX_MLP_LAYERS 4
#define NTBC_HIDDEN_WIDTH 64

/* Returns the calling thread's message for the last failed call ("" if none). */
const char* ntbc_last_error(void);

/* ABI version; bumps whenever a struct layout or signature changes. */
int ntbc_abi_version(void);

/* ------------------------------------------------------------------------- */
/* BC1 / BC4 codec                                                            */
/* ------------------------------------------------------------------------- */

/*
 * Reference BC encoder (stands in for the Compressonator encoder that produces
 * the training targets and the "Ref. BC" quality bar, Sec. 3.2 and Sec. 4.1).
 * BC1: principal-axis range fit (integer covariance, 8 FP64 power iterations,
 * extreme-projection texels as endpoints), RGB565 quantisation, exhaustive
 * per-texel code choice, colour0 > colour1. BC4: best of the 8-value mode over
 * [min, max] and the 6-value mode over the texels other than 0 and 255.
 * Deterministic; bit-exact with the CPU oracle.
 *   fmt     NTBC_BC1, NTBC_BC4, or the compositions NTBC_BC3 / NTBC_BC5
 *   texels  device, w*h*C bytes, row-major, C = 3 (BC1), 1 (BC4), 4 (BC3), 2 (BC5)
 *   blocks  device, (w/4)*(h/4)*8 bytes (BC1, BC4) or *16 (BC3, BC5), written
 */
ntbc_status bc_reference_encode(int fmt, const uint8_t* texels, int w, int h,
                                uint8_t* blocks, void* stream);

/*
 * The same encoder followed by up to `refine` (0..16) least-squares refinement steps, our
 * reading of the "refine steps" Sec. 4.1 mentions for Compressonator: the endpoints that
 * minimise the block's squared error for its current codes (closed-form 2x2 normal
 * equations), re-quantised with round-half-up in exact integer arithmetic, the codes
 * re-chosen (BC4 keeps its mode), kept while the squared error strictly falls. Bit-exact
 * with the oracle. refine = 0 is bc_reference_encode.
 */
ntbc_status bc_reference_encode_refined(int fmt, const uint8_t* texels, int w, int h, int refine,
                                        uint8_t* blocks, void* stream);

/*
 * Decoder (the "existing BC decompression" of Sec. 4.4): blocks -> texels with
 * the integer palette (interpolants rounded to nearest; BC1 colour0 <= colour1
 * selects the 3-colour mode, BC4 r0 <= r1 the 6-value mode with 0 and 255).
 *   blocks  device, (w/4)*(h/4)*8 (BC1, BC4) or *16 (BC3, BC5) bytes
 *   texels  device, w*h*C bytes (C as for the encoder), written
 */
ntbc_status bc_decode(int fmt, const uint8_t* blocks, int w, int h,
                      uint8_t* texels, void* stream);

/*
 * Steps a6-a8 of NTBC inference on given network outputs (Sec. 3.2, Fig. NTBC
 * (a)): quantise predicted endpoints (floor(e*31+0.5), G *63, BC4 *255, FP32),
 * order BC1 colour0 > colour1 by swapping (equal: all codes 0) or take the BC4
 * mode from r0 > r1, build the integer palette / 255, pick per texel the code of
 * least squared FP32 distance (ties: lowest code), pack.
 *   e_hat   device float [n][2*C]  (e0 then e1; C = 3 for BC1, 1 for BC4)
 *   c_hat   device float [n][16][C] predicted texel colours in [0, 1]
 *   blocks  device, n*8 bytes, written
 */
ntbc_status ntbc_outputs_to_bc(int fmt, const float* e_hat, const float* c_hat, int n,
                               uint8_t* blocks, void* stream);

/* ------------------------------------------------------------------------- */
/* Model                                                                      */
/* ------------------------------------------------------------------------- */

/*
 * Architecture of one NTBC model (Sec. 3.2, Sec. 3.4, Sec. 4.1): an endpoint
 * network over block coordinates and a colour network over texel coordinates,
 * each a multi-resolution 2D feature grid (dense res x res x features per level,
 * bilinear, corner aligned) followed by an MLP with `hidden_layers` hidden layers
 * of 64 units and sigmoid outputs. The textures of the material share one model
 * (aggressive packaging); the conservative packaging is two models.
 */
typedef struct {
    int width, height;                     /* texels of every texture of the material */
    int n_textures;                        /* 1..NTBC_MAX_TEXTURES */
    int formats[NTBC_MAX_TEXTURES];        /* NTBC_BC1 / NTBC_BC4, material order */
    int color_levels;                      /* 1..NTBC_MAX_LEVELS */
    int color_res[NTBC_MAX_LEVELS];        /* per-level resolution, >= 2 */
    int endpoint_levels;
    int endpoint_res[NTBC_MAX_LEVELS];
    int features;                          /* features per level (2) */
    int hidden_layers;                     /* 1..3 */
    int hidden_width;                      /* must be 64 */
    int activation;                        /* NTBC_ACT_SELU / NTBC_ACT_RELU */
} ntbc_model_desc;

typedef struct { size_t offset, count; } ntbc_span;   /* in floats */

/*
 * Flat FP32 parameter layout: colour-grid levels (each [res][res][features],
 * row = y), endpoint-grid levels, colour MLP (per layer W [out][in] then b
 * [out]), endpoint MLP. in/out: MLP input (features*levels) and output sizes
 * (colour 3 per BC1 + 1 per BC4 texture; endpoint twice that: e0 then e1 per
 * texture, in material order).
 */
typedef struct {
    size_t total;
    ntbc_span color_grid[NTBC_MAX_LEVELS];
    ntbc_span endpoint_grid[NTBC_MAX_LEVELS];
    ntbc_span color_w[NTBC_MAX_MLP_LAYERS], color_b[NTBC_MAX_MLP_LAYERS];
    ntbc_span endpoint_w[NTBC_MAX_MLP_LAYERS], endpoint_b[NTBC_MAX_MLP_LAYERS];
    int in_color, out_color, in_endpoint, out_endpoint;
    size_t grid_floats;                    /* colour + endpoint grid floats (a prefix) */
} ntbc_layout;

/* Host-only: validate desc and fill the layout. No device work. */
ntbc_status ntbc_model_layout(const ntbc_model_desc* desc, ntbc_layout* out);

/*
 * Grid level resolutions res_l = floor(n_min * (n_max/n_min)^(l/(levels-1)) + 0.5)
 * (geometric ladder from the coarsest to the finest resolution, Sec. 3.4).
 * Host-only. out: host int[levels].
 */
ntbc_status ntbc_level_resolutions(int levels, int n_min, int n_max, int* out);

typedef struct ntbc_model ntbc_model;      /* opaque, library-owned device state */

/* Allocate a model (FP32 master parameters on the current device, zeroed). */
ntbc_status ntbc_model_create(const ntbc_model_desc* desc, ntbc_model** out);
void ntbc_model_free(ntbc_model* model);
/* Device pointer and float count of the FP32 master parameters (layout above). */
ntbc_status ntbc_model_params(ntbc_model* model, float** params, size_t* count);
/*
 * Copy `count` floats (must equal layout.total) of FP32 master parameters from
 * device `src` into the model, or from the model into device `dst`. Async.
 */
ntbc_status ntbc_model_set_params(ntbc_model* model, const float* src, size_t count, void* stream);
ntbc_status ntbc_model_get_params(const ntbc_model* model, float* dst, size_t count, void* stream);

/*
 * Build the inference form (Sec. 3.3): with grid_bits 8 or 4 every grid level is
 * quantised as in QAT (range [min(0,min), max(0,max)], s = range/(2^b-1),
 * z = round(-alpha/s), q = clamp(round(r/s)+z), FP32 decisions) and stored as one
 * code per byte plus (s, z) per level; grid_bits 0 keeps FP32 grids.
 * weight_prec NTBC_PREC_FP16 / NTBC_PREC_FP16_FAST rounds MLP weights and biases to
 * half precision (round to nearest even) and prepares the tensor-core weight image;
 * NTBC_PREC_FP8 quantises them to E4M3 with per-layer power-of-two scales (layers in
 * the order colour 0.., endpoint 0..; a layer's weights and bias share its scale);
 * NTBC_PREC_FP8_MMA does the same and then calibrates the per-layer activation scales
 * on the exported grids (one small kernel; the calibration sample is described with
 * the precision modes); NTBC_PREC_FP32 keeps them.
 */
ntbc_status ntbc_model_export(ntbc_model* model, int grid_bits, int weight_prec, void* stream);

/*
 * Read back the exported grid: codes (device, grid_floats bytes, same element
 * order as the grid part of the layout), scales and zeros (device float
 * [color_levels + endpoint_levels]).
 */
ntbc_status ntbc_model_exported_grid(const ntbc_model* model, uint8_t* codes, float* scales,
                                     float* zeros, void* stream);

/* Size in bytes of the stored model blob of the current export (host-only query). */
ntbc_status ntbc_model_blob_size(const ntbc_model* model, size_t* size);

/*
 * Stored model blob (the on-disk form the paper loads at texture-load time):
 * exported grid codes (8-bit: one per byte; 4-bit: two per byte, the lower-indexed
 * code in the low nibble; or the FP32 grid), per-level (s, z), MLP weights in the
 * export precision (FP8: 2 * NTBC_MAX_MLP_LAYERS int32 weight exponents, then for
 * NTBC_PREC_FP8_MMA as many activation exponents, then one E4M3 code per parameter). A 4-bit blob is packed and unpacked on the device (one kernel
 * each way). Loading a blob whose header is not this ABI version, describes another
 * model or names an unknown grid width / precision returns NTBC_EINVAL. ntbc_model_save copies device -> host `blob` (host,
 * blob_size bytes; synchronises the stream); ntbc_model_load copies host `blob`
 * (pinned host memory recommended) -> the model's device buffers, asynchronously.
 */
ntbc_status ntbc_model_save(const ntbc_model* model, uint8_t* blob, size_t size, void* stream);
ntbc_status ntbc_model_load(ntbc_model* model, const uint8_t* blob, size_t size, void* stream);

/* ------------------------------------------------------------------------- */
/* Inference (Sec. 3.2, Fig. NTBC (a); Sec. 4.4)                              */
/* ------------------------------------------------------------------------- */

/*
 * NTBC inference to BC blocks for every texture of the model's material, in one
 * fused kernel: grid lookup + dequantisation, endpoint MLP per block, colour MLP
 * per texel, endpoint quantisation, per-texel argmax of -||c_hat - p_n||, index
 * packing and 8-byte block stores. Uses the exported form (ntbc_model_export). One
 * launch, or on the tensor-core path two when a full grid's last round is partial (that
 * round's blocks in half-size work units, chained by programmatic dependent launch;
 * ntbc_infer_plan tells which). Enqueued on `stream`; asynchronous.
 *   blocks_out  host array of n_textures DEVICE pointers, each (w/4)*(h/4)*8 bytes
 */
ntbc_status ntbc_infer_to_bc(const ntbc_model* model, uint8_t* const* blocks_out, void* stream);

/*
 * The same inference with the blocks delivered to HOST memory: the material's blocks are
 * produced in `chunks` (1..16) consecutive ranges of whole 128-block work units, and each
 * range is copied device -> host (one copy per texture, on a copy stream the model keeps)
 * while the next range is computed, so the transfer hides behind the inference. On the
 * tensor-core path each range after the first is a programmatic dependent launch, which may
 * start while the previous range's last CTAs finish (the ranges write disjoint blocks).
 *   host_out  host array of n_textures HOST pointers, each (w/4)*(h/4)*8 bytes; pinned
 *             memory lets the copies overlap the compute (pageable memory still works)
 * Everything is ordered before later work on `stream`: the blocks are in host_out once
 * `stream` has been synchronised. The first call allocates a device staging area of the
 * material's block bytes, the block ids 0..n-1, a stream and events, all kept by the model
 * until ntbc_model_free; calls on one model must not overlap.
 */
ntbc_status ntbc_infer_to_host(ntbc_model* model, uint8_t* const* host_out, int chunks, void* stream);

/*
 * The launch plan of ntbc_infer_to_bc for an exported model (host-only query; no launch):
 * launches = kernel launches per call (1; or 2 on the tensor-core path when a full grid's last
 * round is partial: its blocks go to a chained launch of half-size work units),
 * unit_blocks = blocks per work unit (128 or 64; 0 for the FP32 SIMT kernel),
 * units_in_flight = work units one launch runs at once (warpgroups x CTAs; 0 for FP32).
 * NTBC_EINVAL for a null argument or a model that has not been exported.
 */
ntbc_status ntbc_infer_plan(const ntbc_model* model, int* launches, int* unit_blocks, int* units_in_flight);

/*
 * Failure-path check of the bounded device waits: one thread polls an mbarrier that nothing
 * will complete, with the wait loop of the tensor-core kernels limited to `polls` polls
 * (1 .. the kernels' own limit, 2^18, about one second). Returns NTBC_ETIMEOUT when the wait gave up (the
 * expected outcome; the GPU context stays usable) and the wait's duration in *seconds
 * (optional). Synchronises `stream`.
 */
ntbc_status ntbc_wait_probe(long long polls, double* seconds, void* stream);

/*
 * Measurement utility; the paper has no counterpart. The exp2 throughput of the device
 * (ex2.approx results per second over all SMs: 8 independent dependency chains per thread,
 * 8 CTAs of 256 threads per SM), the MUFU peak against which the inference kernel's roofline
 * is reported (its SELU and sigmoid evaluate one exp2 per unit). About 10 ms of device work;
 * allocates a small scratch buffer; synchronises `stream`.
 */
ntbc_status ntbc_ex2_rate_probe(double* ex2_per_s, void* stream);

/*
 * The same with a block stride per texture: block b of texture t is written at
 * blocks_out[t] + b * block_stride[t] (a positive multiple of 8; NULL means 8 for all). With
 * stride 16 two textures of the model fill one 16-byte-block texture: a BC4 alpha texture
 * at offset 0 and a BC1 colour texture at offset 8 make BC3; two BC4 textures make BC5.
 */
ntbc_status ntbc_infer_to_bc_strided(const ntbc_model* model, uint8_t* const* blocks_out,
                                     const int* block_stride, void* stream);

/*
 * Raw network outputs (pre-quantisation) of the exported model at given blocks:
 *   block_ids  device int32 [n]
 *   e_hat      device float [n][out_endpoint]
 *   c_hat      device float [n][16][out_color]  (texel i = 4y + x of each block)
 * n = 0 returns NTBC_OK without touching the pointers (which may then be NULL).
 */
ntbc_status ntbc_forward(const ntbc_model* model, const int32_t* block_ids, int n,
                         float* e_hat, float* c_hat, void* stream);

/*
 * Batched load-time inference (Sec. 4.4: inference runs once per material when it is
 * loaded): many materials, each with its own model, decoded to BC blocks by one call.
 * Every model must be exported with a tensor-core precision (not NTBC_PREC_FP32), and the
 * output ranges of all materials and textures must be disjoint (they are written
 * concurrently; NTBC_EINVAL otherwise). Two modes:
 *   NTBC_BATCH_CHAINED (ntbc_batch_create's mode) one launch of the single-material kernel
 *                      per material, largest material first, each after the first a
 *                      programmatic dependent launch: it may start as soon as every CTA of
 *                      the previous launch is resident, so its CTAs take the SMs the previous
 *                      material leaves at its tail. Materials may mix precisions.
 *   NTBC_BATCH_QUEUE   one persistent launch whose CTAs take work from a device queue of
 *                      CTA-units (one work unit per warpgroup), the materials queued largest
 *                      first; all models must be exported for the same tensor-core kernel
 *                      (NTBC_PREC_FP16 / NTBC_PREC_FP8, NTBC_PREC_FP16_FAST, or
 *                      NTBC_PREC_FP8_MMA). A claim outside the queue does no work; after 2^16
 *                      of them a CTA gives up and the launch reports NTBC_ETIMEOUT through
 *                      ntbc_batch_times (host-side fault injection NTBC_FAULT=ticket starts
 *                      the counter negative to test this).
 *   ntbc_batch_create(_mode)  models: host array of n models; blocks_out: host array of n
 *                      host arrays, each holding that material's per-texture DEVICE outputs
 *                      (8-byte aligned, n_blocks * 8 bytes each). Plans the launches
 *                      (allocates; waits for all work on the device, so models exported on
 *                      any stream are complete; not capturable). An unknown mode is
 *                      NTBC_EINVAL.
 *   ntbc_batch_infer   one reset of the batch's counters, then the launches on `stream`; may
 *                      be captured in a CUDA graph and replayed.
 *   ntbc_batch_times   synchronises `stream`; ms (host double[n], in the order of `models`)
 *                      = each material's completion time after the start of the batch's first
 *                      launch (device global timer); NTBC_ETIMEOUT if a bounded wait or the
 *                      bounded claim loop gave up.
 */
enum { NTBC_BATCH_CHAINED = 0, NTBC_BATCH_QUEUE = 1 };
typedef struct ntbc_batch ntbc_batch;
ntbc_status ntbc_batch_create(const ntbc_model* const* models, int n, uint8_t* const* const* blocks_out,
                              ntbc_batch** out);
ntbc_status ntbc_batch_create_mode(const ntbc_model* const* models, int n, uint8_t* const* const* blocks_out,
                                   int mode, ntbc_batch** out);
ntbc_status ntbc_batch_infer(ntbc_batch* batch, void* stream);
ntbc_status ntbc_batch_times(const ntbc_batch* batch, double* ms, void* stream);
void ntbc_batch_free(ntbc_batch* batch);

/* ------------------------------------------------------------------------- */
/* Training (Sec. 3.2 losses and straight-through argmax; Sec. 3.3 QAT;        */
/* Sec. 3.4 Adam + schedule)                                                 */
/* ------------------------------------------------------------------------- */

typedef struct {
    int width, height, n_textures;
    int formats[NTBC_MAX_TEXTURES];
    const uint8_t* texels[NTBC_MAX_TEXTURES];       /* device, source textures */
    const uint8_t* ref_blocks[NTBC_MAX_TEXTURES];   /* device, reference BC blocks (targets) */
} ntbc_material;

typedef struct {
    long steps;                 /* main-phase steps S */
    int batch_texels;           /* texels per step (multiple of 16: whole blocks) */
    float qat_fraction;         /* extra ceil(fraction*S) QAT steps; 0 disables QAT */
    int grid_bits;              /* QAT bit width (8 or 4) */
    float lr_grid, lr_mlp;      /* peak learning rates (0.01, 0.005) */
    float temperature;          /* softmax temperature T (0.01) */
    int warmup;                 /* linear warm-up steps (10) */
    uint64_t seed;              /* Philox key of the batch sampler */
    int precision;              /* NTBC_TRAIN_FP32 or NTBC_TRAIN_BF16 (see below) */
} ntbc_train_config;

/*
 * Training arithmetic:
 *   NTBC_TRAIN_FP32  layer-by-layer FP32 kernels (activations in HBM, feature-major)
 *   NTBC_TRAIN_BF16  one fused tensor-core pass per network: BF16 MMA operands (features,
 *                    activations, weights, deltas) with FP32 accumulation in TMEM; losses,
 *                    sigmoid, straight-through argmax, grid gather / scatter and Adam in FP32.
 *                    The endpoint network's forward splits each operand into BF16 hi + lo
 *                    parts (~16 significant bits): its outputs set the palettes that the
 *                    straight-through softmax of App. A scores at temperature T, which
 *                    amplifies an output error 1/T. Activations live on chip for one
 *                    128-sample tile, so device memory does not grow with the batch.
 *                    Gradients within about 4e-2 of FP64 at T = 0.01 (colour network), 1.5e-2
 *                    (endpoint network).
 */
enum { NTBC_TRAIN_FP32 = 0, NTBC_TRAIN_BF16 = 1 };

/*
 * Losses and gradients of one training step on the given blocks (all 16
 * texels of each), for the current FP32 master parameters.
 *   block_ids  device int32 [n_blocks]
 *   qat_bits   0 (float grids) or the QAT width (fake-quantised grids, STE)
 *   precision  NTBC_TRAIN_FP32 or NTBC_TRAIN_BF16
 *   grads      device float [layout.total], overwritten with d loss / d params
 *              (endpoint parameters: of L_e + L_cd; colour: of L_c + L_cd)
 *   losses     device float [6]: L_e, L_cd(endpoint), L_c, L_cd(colour),
 *              L_endpoint, L_color
 */
ntbc_status ntbc_train_grads(ntbc_model* model, const ntbc_material* mat, const int32_t* block_ids,
                             int n_blocks, int qat_bits, float temperature, int precision,
                             float* grads, float* losses, void* stream);

/*
 * Forward and vector-Jacobian product of the raw network outputs on the FP32 master
 * parameters: the training forward (grid lookup, fake quantisation of the grids when
 * qat_bits > 0, MLPs, sigmoid) and the hand-written backward (weight and bias
 * gradients, input gradients, grid scatter-add, straight-through quantiser) that the
 * losses of Sec. 3.2 drive, here driven by an arbitrary upstream gradient. This is the
 * differentiable-function form of the network for gradient checks and for use inside
 * other losses; every call recomputes the activations from the parameters (nothing is
 * kept between a forward and a later backward).
 *   block_ids  device int32 [n_blocks] (repeats allowed)
 *   g_e, g_c   device float, upstream d f / d e_hat [n_blocks][out_endpoint] and
 *              d f / d c_hat [n_blocks][16][out_color], or both NULL (forward only)
 *   grads      device float [layout.total], overwritten with sum g . d outputs / d params
 *              (may be NULL when g_e, g_c are NULL)
 *   e_hat, c_hat  device float outputs in the layout of ntbc_forward, or NULL
 */
ntbc_status ntbc_vjp(ntbc_model* model, const int32_t* block_ids, int n_blocks, int qat_bits,
                     const float* g_e, const float* g_c, float* grads, float* e_hat, float* c_hat,
                     void* stream);

/*
 * Steps [first_step, last_step) of the encode that ntbc_train runs in one call (the schedule of
 * `cfg`: cfg->steps main steps, then ceil(qat_fraction * steps) QAT steps, the LR warm-up and
 * cosine over all of them, batches sampled by (seed, step)). first_step = 0 starts a fresh
 * encode (Adam moments zeroed); first_step > 0 continues from the model's current parameters
 * and Adam moments, as left by the previous range or by ntbc_checkpoint_load, so an encode can
 * be split at any step and resumed in another process. Synchronises the stream at the end;
 * losses_out (host float[6], may be NULL): the last step's losses; NTBC_ENONFINITE if they are
 * not finite. A resumed encode matches an uninterrupted one up to the rounding order of the
 * grid scatter's floating-point atomics (two uninterrupted encodes differ as much).
 */
ntbc_status ntbc_train_range(ntbc_model* model, const ntbc_material* mat, const ntbc_train_config* cfg,
                             long first_step, long last_step, float* losses_out, void* stream);

/*
 * Training checkpoint of a model: its description, the step a resumed encode starts at, the FP32
 * master parameters and both Adam moments (3 x layout.total floats after a small header).
 * ntbc_checkpoint_save copies device -> host `buf` (host, ntbc_checkpoint_size bytes) and
 * synchronises `stream`; ntbc_checkpoint_load copies it back into a model of the same
 * description (NTBC_EINVAL otherwise, or for a header of another ABI version), synchronises, and
 * returns the step to resume at in *next_step (optional). The resumed encode is then
 * ntbc_train_range(model, mat, cfg, next_step, total, ...) with the same cfg.
 */
ntbc_status ntbc_checkpoint_size(const ntbc_model* model, size_t* size);
ntbc_status ntbc_checkpoint_save(ntbc_model* model, uint8_t* buf, size_t size, void* stream);
ntbc_status ntbc_checkpoint_load(ntbc_model* model, const uint8_t* buf, size_t size, long* next_step, void* stream);

/*
 * Allocation-free variant of ntbc_train_grads. The paper has no counterpart.
 * For callers that cannot allocate device memory: an engine's texture-streaming
 * thread working inside a fixed, pre-reserved VRAM budget, or a real-time thread
 * that cannot afford the device-wide synchronisation of cudaMalloc. It calls no
 * cudaMalloc / cudaFree or other allocating routine; its scratch is a file-scope
 * device array of NTBC_NOALLOC_MAX_BLOCKS blocks' worth (about 3.3 MB) that every
 * GPU loading the library holds until the process exits.
 *   desc, params  model description (host) and FP32 parameters (device, layout of
 *                 ntbc_model_layout); block_ids, qat_bits, temperature, grads and
 *                 losses as in ntbc_train_grads, with `losses` required. There is no
 *                 precision argument: this call always runs the FP32 layer-by-layer
 *                 kernels (NTBC_TRAIN_FP32), the same launches ntbc_train_grads makes
 *                 for that precision.
 *   n_blocks      1..NTBC_NOALLOC_MAX_BLOCKS, else NTBC_EINVAL before any launch.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call before
 * any stream capture. All calls share the one array: calls whose work overlaps
 * on the GPU (other streams, other threads) race on it and must be serialised
 * by the caller. Gradients and loss accumulators are cleared on every call.
 */
#define NTBC_NOALLOC_MAX_BLOCKS 128
ntbc_status ntbc_train_grads_noalloc(const ntbc_model_desc* desc, const float* params, const ntbc_material* mat,
                                     const int32_t* block_ids, int n_blocks, int qat_bits, float temperature,
                                     float* grads, float* losses, void* stream);

/*
 * One dense Adam step (beta 0.9/0.999, eps 1e-15, bias correction) on the FP32
 * master parameters with learning rate lr_grid / lr_mlp scaled by the warm-up +
 * cosine schedule at `step` of `total_steps`. Adam moments are library-owned
 * and start at zero at step 0.
 */
ntbc_status ntbc_adam_step(ntbc_model* model, const float* grads, long step, long total_steps,
                           const ntbc_train_config* cfg, void* stream);

/*
 * Philox4x32-10 batch sampler: ids[i] = (word * n_blocks) >> 32 with word
 * (i mod 4) of philox(counter = (i/4, step, 0, 0), key = (seed lo, seed hi)).
 *   ids  device int32 [n]
 */
ntbc_status ntbc_sample_blocks(uint64_t seed, long step, int n, int n_blocks, int32_t* ids, void* stream);

/*
 * Full encode (Fig. NTBC (b)): S main steps then ceil(qat_fraction*S) QAT steps,
 * each sampling batch_texels/16 blocks, computing gradients and taking an Adam
 * step, all on device; the per-step launches are captured once in a CUDA graph.
 * The model's parameters must be initialised (ntbc_model_params) by the caller.
 * Synchronises the stream at the end. losses_out: host float[6] of the last
 * step (may be NULL). NTBC_ENONFINITE if the last loss is not finite.
 */
ntbc_status ntbc_train(ntbc_model* model, const ntbc_material* mat, const ntbc_train_config* cfg,
                       float* losses_out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* NTBC_H */
