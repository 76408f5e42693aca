/*
 * hyena.h -- C ABI of the GB300 library for homomorphically encrypted
 * convolution with Walsh-Hadamard output-channel packing ("Hyena",
 * arXiv 2311.12519).
 *
 * Problem statement (Sec. 2.2, Sec. 3): a client encrypts the input of a
 * convolution layer under BFV (Sec. 2.3); the cloud, holding integer filter
 * weights, computes the encrypted convolution with the padded convolution of
 * Sec. 2.4, packs pairs of output channels per ciphertext with the
 * Walsh-Hadamard decomposition of Eq. 1, defers modular reduction (Sec.
 * 3.2.2) and uses parameters chosen as in Sec. 3.2.1; the client decrypts.
 *
 * Conventions for every call:
 *  - Return value: HE_OK (0) or an HE_E* code; he_last_error() then returns
 *    a thread-local message.  No C++ exception crosses this boundary.
 *  - Opaque handles are created and destroyed only by this library.
 *  - Host buffers and device buffers passed in are owned by the caller; the
 *    library reads and writes them only for the duration of the call (for
 *    device calls: of the work enqueued on the given stream).  The library
 *    owns the device copies of keys and tables held inside a plan.
 *  - Ciphertext arrays are uint64 [n_ct][2][L][N]: polynomial c0/c1, RNS limb
 *    q_k, coefficient; every word is a canonical residue in [0, q_k), in
 *    coefficient form.
 *  - Device pointers must be 16-byte aligned.  Calls on a stream are
 *    asynchronous unless stated otherwise.
 *  - Host-only calls (parameters, keys, encrypt, decrypt, layout) need no GPU.
 */
#ifndef HYENA_H
#define HYENA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HE_OK 0
#define HE_EINVAL 1       /* bad argument, unsupported shape, null pointer */
#define HE_ENOMEM 2       /* host or device allocation failed */
#define HE_ECUDA 3        /* a CUDA runtime call failed */
#define HE_ENOISE 4       /* the noise estimate exceeds the decryption margin */
#define HE_ETIMEOUT 5     /* a bounded device wait gave up */
#define HE_EMISSINGKEY 6  /* a plan needs a Galois key that was not generated */

#define HE_MAX_LIMBS 8

typedef struct he_params he_params;   /* encryption parameters + host tables */
typedef struct he_seckey he_seckey;   /* ternary secret key (client side) */
typedef struct he_galkeys he_galkeys; /* key-switching keys for Galois elements */
typedef struct he_plan he_plan;       /* one convolution layer, device resident */

/* Thread-local description of the last failure in this thread ("" if none). */
const char* he_last_error(void);

/* ------------------------------------------------------------------ */
/* Parameters (Sec. 3.2.1)                                            */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t N;              /* ring degree, power of two in [1024, 16384] */
    uint32_t L;              /* RNS limbs q_1..q_L, 1 <= L <= HE_MAX_LIMBS */
    uint32_t limb_bits;      /* q_i are the largest primes < 2^limb_bits, = 1 mod 2N (30..54; 0 -> 50) */
    uint32_t t_bits;         /* if t == 0: t = largest prime < 2^t_bits, = 1 mod 2N (0 -> 20) */
    uint64_t t;              /* plaintext modulus p; must be prime and = 1 mod 2N; 0 -> from t_bits */
    uint32_t decomp_bits;    /* key-switching base 2^w; 0 -> largest w whose noise estimate fits */
    uint32_t k_max;          /* search range [1, k_max] for k (0 -> 32) */
    uint32_t est_mac_terms;  /* for decomp_bits == 0: largest C_in * kh^2 the parameters must carry */
    uint32_t est_weight_max; /* for decomp_bits == 0: largest |weight| (0 -> 8) */
} he_param_req;

typedef struct {
    uint32_t N, L;
    uint32_t w;              /* decomposition bits */
    uint32_t l;              /* digits per limb = ceil(bits(q_max) / w) */
    uint64_t t;              /* plaintext modulus p */
    uint64_t zeta;           /* slot root: smallest primitive 2N-th root of unity mod t */
    uint64_t h;              /* h_{p,n} in [0, t): coefficient of the [1,-1] plaintext */
    uint64_t k;              /* the k of Sec. 3.2.1 */
    int64_t kh;              /* centred [k h]_t: the two non-zero coefficients of [k,-k] */
    double log2_delta;       /* log2 floor(q / t) */
    double est_noise_log2;   /* noise estimate behind the choice of w (log2) */
    uint64_t q[HE_MAX_LIMBS];
    uint64_t k4;             /* the k of c_n = 4 packing: in [1, min(t - 1, 2^20)], minimising
                                k + sum |[k a]_t| over the non-zero coefficients a of the three
                                +-1 patterns of the 4 x 4 Walsh-Hadamard basis (ties -> smallest) */
} he_param_info;

/* Runs the selection of Sec. 3.2.1: primes p = q_i = 1 (mod 2N), h_{p,n}, the
 * k in [1, k_max] minimising |[k h]_p| (ties -> smallest), then the largest
 * decomposition base whose estimated noise stays below a quarter of
 * floor(q/t).  Host only.  Errors: HE_EINVAL (shape, t not prime or not
 * = 1 mod 2N), HE_ENOISE (no base fits). */
int he_params_create(const he_param_req* req, he_params** out);
int he_params_info(const he_params* p, he_param_info* out);
void he_params_destroy(he_params* p);

/* ------------------------------------------------------------------ */
/* Keys (client side, host)                                           */
/* ------------------------------------------------------------------ */
/* Ternary secret key from a seed (SplitMix64 stream, tag 1). */
int he_keygen(const he_params* p, uint64_t seed, he_seckey** out);
/* Copies the secret key's coefficients (int64[N], values in {-1,0,1}). */
int he_seckey_export(const he_seckey* sk, int64_t* coeffs);
void he_seckey_destroy(he_seckey* sk);

/* Key-switching keys for n Galois elements (odd, in [3, 2N)).  Key for
 * element g, digit (i,j): (b, a) with b = -a s + e + 2^(w j) [i = k] sigma_g(s)
 * mod q_k (Sec. 2.3, rotation; BV-style gadget over the RNS limbs).
 * Seeded streams: tag 4 (a) and tag 5 (e) per (g, digit).  Host only. */
int he_galois_keys(const he_params* p, const he_seckey* sk, const uint32_t* galois, int n, uint64_t seed,
                   he_galkeys** out);
/* Copies the key of Galois element g: uint64 [L*l][2][L][N], coefficient form. */
int he_galkeys_export(const he_galkeys* gk, uint32_t galois, uint64_t* out);
void he_galkeys_destroy(he_galkeys* gk);

/* ------------------------------------------------------------------ */
/* Layer description and slot layout (Sec. 2.4, Sec. 3.1)             */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t C_in, C_out;    /* channels; depthwise needs C_in == C_out */
    uint32_t H, W;           /* input height and width */
    uint32_t kh;             /* odd square kernel size (1, 3, 5, 7); padding is (kh-1)/2 */
    uint32_t stride;         /* 1 or 2 */
    uint32_t depthwise;      /* 0 or 1 */
    uint32_t n_images;       /* images packed into the same ciphertexts (same client key) */
    uint32_t c_n;            /* channels per ciphertext: 2 (Hyena packing), 1 (padded conv) or 4
                                (Sec. 3.1's 4 x 4 Walsh-Hadamard basis: channel 4j + c of ciphertext
                                j in slot row c >> 1 at slot parity c & 1, N/4 block positions per
                                row; rotations 2o and 2o +- 1 per tap offset o; CUDA-core MAC only,
                                no polyphase) */
    uint32_t tile_h, tile_w; /* interior tile size, or both 0 for the default: the whole image if its
                                padded block fits half a ring, else full-width strips, else square
                                tiles, each as large as fits.  Given tiles must fit the image, be
                                multiples of the stride unless they span the image, and their padded
                                block (tile_h + kh - 1)(tile_w + kh - 1) must fit N/2 slots (N/4
                                positions with c_n = 4). */
    uint32_t polyphase;      /* 3x3 stride-2 layers only: 1 packs the four phase planes
                                in[2u + a][2v + b] of the input (channel (2a + b) Cp + c, Cp = C_in
                                rounded up to c_n) and runs the layer as a stride-1 layer on them,
                                with taps at offsets -1 and 0 only (the paper leaves stride open,
                                Sec. 2.4); tiles then refer to the ceil(H/2) x ceil(W/2) planes.
                                0 computes the stride-1 result and keeps every second position. */
} he_conv_desc;

typedef struct {
    uint32_t P;              /* padding (kh-1)/2 */
    uint32_t T_h, T_w;       /* interior tile size */
    uint32_t W_b;            /* block row width T_w + 2P: tap (dy,dx) = rotation by dy W_b + dx */
    uint32_t block_slots;    /* (T_h + 2P) W_b */
    uint32_t blocks_per_row; /* tiles held by one slot row (N/2 slots; N/4 positions with c_n = 4) */
    uint32_t n_ty, n_tx;     /* tiles per image */
    uint32_t units;          /* n_images n_ty n_tx */
    uint32_t row_units;      /* ciphertext columns: units / tiles per ciphertext, rounded up */
    uint32_t in_groups, out_groups; /* ceil(C / c_n) */
    uint32_t n_ct_in, n_ct_out;     /* row_units * groups */
    uint32_t Ho, Wo;         /* output size */
    uint32_t n_galois;       /* distinct non-identity Galois elements the layer rotates by */
    uint64_t scale;          /* output = scale * conv (mod t): 2k with c_n = 2, 4 k4 with c_n = 4, 1 with c_n = 1 */
} he_layout;

/* Tiles the zero-padded input into blocks that fit one slot row; host only. */
int he_layout_for_layer(const he_params* p, const he_conv_desc* d, he_layout* out);
/* Writes the layer's Galois elements (ascending) into galois[cap]; *n = count. */
int he_layer_galois(const he_params* p, const he_conv_desc* d, uint32_t* galois, int cap, int* n);

/* ------------------------------------------------------------------ */
/* Client encryption / decryption (host, for tests and the e2e path)  */
/* ------------------------------------------------------------------ */
/* act: int64 [n_images][C_in][H][W] with values in [0, t).  ct_out: uint64
 * [n_ct_in][2][L][N].  Ciphertext c uses the seeded streams (seed, tag 2/3, c). */
int he_encrypt_image(const he_params* p, const he_seckey* sk, const he_conv_desc* d, const int64_t* act,
                     uint64_t seed, uint64_t* ct_out);
/* ct: uint64 [n_ct_out][2][L][N].  out: int64 [n_images][C_out][Ho][Wo]; with
 * unscale != 0 the values are multiplied by scale^-1 mod t (then equal conv mod t). */
int he_decrypt_image(const he_params* p, const he_seckey* sk, const he_conv_desc* d, const uint64_t* ct,
                     int unscale, int64_t* out);
/* Slot-level helpers: slots int64[N] (flat index row*N/2 + i), one ciphertext. */
int he_encrypt_slots(const he_params* p, const he_seckey* sk, const int64_t* slots, uint64_t seed,
                     uint64_t index, uint64_t* ct_out);
int he_decrypt_slots(const he_params* p, const he_seckey* sk, const uint64_t* ct, int64_t* slots);

/* ------------------------------------------------------------------ */
/* Server side: one convolution layer on the GPU                      */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t mac_groups;     /* CUDA-core MAC: output channel groups per block, 1, 2, 4, 8 or 16
                                (0 -> 8; at most 8 are used with c_n = 2 and 4 with c_n = 4) */
    uint32_t mac_impl;       /* 0 auto (c_n = 4: the CUDA-core MAC; every other value but 1 is
                                HE_EINVAL there), 1 CUDA-core lazy MAC, 2 tensor-core MAC (HE_EINVAL
                                if not exact)
                                in the form auto picks: 4 when the layer's output rows fit one CTA and its
                                input channel groups are not a multiple of 8 or its digit transforms fit
                                64 MB, else 5;
                                3 CUDA-core eager MAC (reduced after every term; for ablations);
                                4 tensor-core MAC that splits the rotated residues into fp16 chunks itself;
                                5 tensor-core MAC on operand images the key switch writes once;
                                6 key switch fused into the tensor-core MAC (rows fitting one CTA only);
                                7 tensor-core MAC on operand images in CTA pairs (tcgen05 cta_group::2,
                                  256 output rows per pair as the MMA's M dimension, 64 slots as N;
                                  HE_EINVAL with tc_rows or tc_cluster set);
                                8 tensor-core MAC on operand images in chunk passes (up to 256 output rows
                                  per CTA, floor(512 / rows) chunks accumulated per pass; HE_EINVAL with
                                  tc_rows or tc_cluster set) */
    uint32_t tc_rows;        /* tensor-core MAC: output rows per CTA, a multiple of 16 up to 96 (0 -> 96) */
    uint32_t tc_cluster;     /* image-form tensor-core MAC: 0 (default) or 2, 4, 8 -- run in clusters of
                                that many CTAs that share each operand image by TMA multicast, each CTA
                                taking a share of the layer's output rows (HE_EINVAL if the layer has too
                                few rows or tc_rows is set) */
    uint32_t reserved[4];
} he_tune;

/* Uploads the layer's Galois keys (NTT form), the Hadamard scalars
 * s0 = v0 + v1, s1 = v0 - v1 of Eq. 1 (int16) and NTT(P_k) of the [k,-k]
 * plaintext to the current CUDA device.  weights: int32
 * [C_out][depthwise ? 1 : C_in][kh][kh], |w| <= 16383.
 * Errors: HE_EINVAL, HE_EMISSINGKEY, HE_ENOISE (estimated output noise too
 * large for these weights), HE_ENOMEM, HE_ECUDA. */
int he_conv_plan(const he_params* p, const he_galkeys* gk, const he_conv_desc* d, const int32_t* weights,
                 const he_tune* tune, he_plan** out);
/* Words (uint64) of the input and output ciphertext arrays and bytes of
 * device workspace one he_conv_forward needs. */
int he_conv_sizes(const he_plan* plan, size_t* in_words, size_t* out_words, size_t* workspace_bytes);
/* Enqueues the layer on `stream` (a cudaStream_t; NULL = legacy default):
 * NTT of inputs and of the base-2^w digits of c1 (hoisting), one key switch
 * per rotation, the lazy channel multiply-accumulate with one reduction per
 * sum, the [k,-k] PMult epilogue, inverse NTT.  d_in / d_out / d_workspace are
 * device pointers sized by he_conv_sizes; d_in is not modified. */
int he_conv_forward(const he_plan* plan, const uint64_t* d_in, uint64_t* d_out, void* d_workspace, void* stream);
/* The same through host buffers: copies h_in to d_in, runs the layer, copies
 * d_out to h_out, and synchronises the stream before returning. */
int he_conv_forward_host(const he_plan* plan, const uint64_t* h_in, uint64_t* h_out, uint64_t* d_in,
                         uint64_t* d_out, void* d_workspace, void* stream);
/* Synchronises the device and returns HE_ETIMEOUT if a bounded wait inside
 * an earlier forward of this plan gave up (the outputs are then invalid). */
int he_conv_status(const he_plan* plan);
/* *mac_impl = 1 (CUDA-core MAC), 3 (eager), or the tensor-core form: 4 (in-kernel conversion),
 * 5 (operand images), 6 (key switch fused), 7 (operand images in CTA pairs) or 8 (operand images
 * in chunk passes) for this plan.  The
 * tensor-core form (fp16 10-bit chunks, fp32 sums of at most 2048 terms per
 * accumulation) is chosen automatically when it is exact: no depthwise,
 * |s| <= 16 and every limb below 2^50 (five chunks). */
int he_conv_info(const he_plan* plan, int* mac_impl);
/* Failure-detection self-test (no paper counterpart).  One CTA waits, through
 * the bounded mbarrier wait every role of the tensor-core MAC uses, on a
 * barrier that nothing arrives at; the wait gives up after its poll limit and
 * reports through a device status word, as a stalled MAC pipeline would.
 * Returns HE_ETIMEOUT when that happened (the expected result; the context
 * stays usable), HE_OK if the wait wrongly completed, or HE_ECUDA. */
int he_selftest_bounded_wait(void* stream);
/* The host-side checks of he_conv_plan alone (layout, scalars, the noise
 * estimate, the tensor-core exactness bound, the tune fields), without keys
 * and without touching the device: HE_OK if he_conv_plan would accept this
 * configuration, else the error it would return (HE_EINVAL, HE_ENOISE). */
int he_conv_check(const he_params* p, const he_conv_desc* d, const int32_t* weights, const he_tune* tune);
/* Device time of one forward of this layer configuration, for tuning and for
 * training the cost model: builds a plan whose key-switching keys and input
 * ciphertexts are uniform residues made on the device (the kernels do the same
 * work on any residues), runs one warm-up and `reps` (1..1000) timed forwards
 * on `stream`, and frees everything.  stage_ms[4] (may be NULL): median times
 * of the input NTTs, key switch, MAC and output NTTs; *total_ms: median of the
 * whole forward.  Errors: as he_conv_plan (HE_ENOISE if the weights would
 * exceed the noise budget), HE_ENOMEM if the buffers do not fit the device. */
int he_conv_time(const he_params* p, const he_conv_desc* d, const int32_t* weights, const he_tune* tune, int reps,
                 void* stream, float* stage_ms, float* total_ms);
void he_plan_destroy(he_plan* plan);

/* Size of the static device scratch used by he_conv_forward_noalloc (32 MiB). */
#define HE_NOALLOC_MAX_SCRATCH_BYTES 33554432u

/* he_conv_forward without any device allocation by anyone.  The paper has no
 * counterpart to this call; it exists for callers that cannot call cudaMalloc
 * or take a workspace buffer from an allocator -- for example code that runs
 * inside a memory pool that already owns all device memory, a service whose
 * device allocations are frozen after start-up, or a latency-bound path where
 * an allocation (which may synchronise the device) is not acceptable.
 *
 * The workspace is a file-scope device array of HE_NOALLOC_MAX_SCRATCH_BYTES
 * that every GPU loading this library holds until the process exits.  Layers
 * whose he_conv_sizes workspace exceeds it are rejected with HE_EINVAL (use
 * he_conv_forward).  The first call on a device looks up the array's device
 * address (cudaGetSymbolAddress) with that device current; make that first
 * call before any stream capture.  The call performs no cudaMalloc, cudaFree
 * or other allocation.  All calls share the one array and it keeps the last
 * call's contents (every word a kernel reads is written earlier in the same
 * call, so nothing needs clearing); calls whose work overlaps on the GPU --
 * on different streams, or from different threads -- race on it.  The
 * caller still owns d_in and d_out; per-stage event timing is not recorded.
 * The plan's device must be current; a call refused for a wrong device or a
 * misaligned pointer touches no device.  The looked-up address is kept per
 * device ordinal for the life of the process, so a cudaDeviceReset after the
 * first call on a device is not supported (the cached address would be stale). */
int he_conv_forward_noalloc(const he_plan* plan, const uint64_t* d_in, uint64_t* d_out, void* stream);

/* ------------------------------------------------------------------ */
/* Batched execution of many layers                                    */
/* ------------------------------------------------------------------ */
/* Layers whose inputs are already encrypted are independent units of work:
 * in private inference every layer input is freshly encrypted by the client
 * (Sec. 2.2), so different layers and images can run together.  A batch runs
 * each stage (input NTT, key switch, channel MAC, output NTT) of all its
 * layers in one launch, so small layers fill the GPU; outputs are identical
 * to he_conv_forward of every plan.  All plans must share one he_params and
 * one device.  The batch keeps pointers to the plans, which must outlive it.
 * A batch caches its CUDA graphs (and, for he_batch_forward_host, a second
 * stream): calls on one batch object must not run concurrently from several
 * host threads.  Plans are read-only after he_conv_plan and may be used by
 * concurrent forwards on different streams with separate workspaces. */
typedef struct he_batch he_batch;
int he_batch_create(const he_plan* const* plans, int n, he_batch** out);
/* The same, with the layers split into waves whose workspaces together fit
 * max_workspace_bytes (first fit, largest workspace first).  Waves run one
 * after another and reuse one workspace region, so a stack larger than the
 * device (VGG-16 on 8 images needs over 100 GB of rotated copies) runs in
 * one call; each wave still launches each stage once for all its layers.  A
 * layer whose own workspace exceeds the limit gets a wave of its own, and the
 * workspace is then that layer's.  he_batch_create is this with no limit. */
int he_batch_create_limited(const he_plan* const* plans, int n, size_t max_workspace_bytes, he_batch** out);
/* *n_waves = the number of waves the batch runs in. */
int he_batch_waves(const he_batch* b, int* n_waves);
/* Device workspace for one he_batch_forward: the largest wave's (layers of a
 * wave get disjoint regions). */
int he_batch_workspace_bytes(const he_batch* b, size_t* bytes);
/* d_in[i], d_out[i]: device buffers of plan i (sizes from he_conv_sizes). */
int he_batch_forward(const he_batch* b, const uint64_t* const* d_in, uint64_t* const* d_out, void* d_workspace,
                     void* stream);
/* The same as a CUDA graph: the first call with a given set of pointers and
 * stream runs the batch once, captures it and instantiates the graph; later
 * calls with the same pointers replay it.  Needs a non-default stream. */
int he_batch_graph_launch(he_batch* b, const uint64_t* const* d_in, uint64_t* const* d_out, void* d_workspace,
                          void* stream);
/* The batch end to end from host memory: copies every layer's input
 * ciphertexts h_in[i] (pinned host memory for asynchronous copies) to d_in[i],
 * runs the batch, copies every output d_out[i] to h_out[i], and synchronises
 * the stream (non-default).  A batch of one wave runs as two halves of about
 * equal input size on `stream` and on a second stream the batch owns, each
 * half its own graph, so that one half's copies overlap the other's kernels.
 * A batch of several waves runs its waves in order on `stream`, while the
 * inputs stream in ahead of them and a finished wave's outputs stream out
 * during the next wave, on two more streams the batch owns; the first wave's
 * input NTTs run one layer at a time, each as soon as its own input has
 * landed, so that only the first layer's copy is exposed.  Outputs equal
 * he_batch_forward's.  Host buffers: on a GB300 with many separately pinned
 * multi-GB buffers live at once, host-to-device copies from them ran at about
 * a quarter of the rate of buffers that are views of one pinned allocation. */
int he_batch_forward_host(he_batch* b, const uint64_t* const* h_in, uint64_t* const* h_out, uint64_t* const* d_in,
                          uint64_t* const* d_out, void* d_workspace, void* stream);
void he_batch_destroy(he_batch* b);

/* ------------------------------------------------------------------ */
/* Single steps, for tests (device pointers, stream-ordered)          */
/* ------------------------------------------------------------------ */
/* In-place negacyclic NTT of n_polys polynomials laid out [n_polys][N];
 * polynomial i is taken mod q_(i mod L).  Output order is bit-reversed:
 * index k holds a(psi_k^(2 rev(k) + 1)), psi_k the library's root for q_k. */
int he_ntt_forward(const he_params* p, uint64_t* d_polys, int n_polys, void* stream);
int he_ntt_inverse(const he_params* p, uint64_t* d_polys, int n_polys, void* stream);
/* HRot (Sec. 2.3) of n_ct ciphertexts by one Galois element through the
 * hoisted key switch; d_ws needs he_rotate_workspace_bytes bytes. */
int he_rotate_workspace_bytes(const he_params* p, int n_ct, size_t* bytes);
int he_rotate(const he_params* p, const he_galkeys* gk, uint32_t galois, const uint64_t* d_in, uint64_t* d_out,
              int n_ct, void* d_ws, void* stream);

/* ------------------------------------------------------------------ */
/* Kernel timing (CUDA events around each launch while enabled)      */
/* ------------------------------------------------------------------ */
#define HE_STAGE_NTT_IN 0   /* forward NTT of inputs and digits */
#define HE_STAGE_KEYSWITCH 1
#define HE_STAGE_MAC 2      /* channel MAC + reduction + PMult epilogue */
#define HE_STAGE_NTT_OUT 3  /* inverse NTT of outputs */
#define HE_N_STAGES 4
typedef struct {
    double ms[HE_N_STAGES];
    uint64_t launches[HE_N_STAGES];
} he_stage_times;
/* Enable (1) or disable (0) per-stage event timing for later forwards. */
int he_profile_enable(int on);
/* Synchronises the recorded events and accumulates them into *out; resets. */
int he_profile_collect(he_stage_times* out);

#ifdef __cplusplus
}
#endif
#endif
