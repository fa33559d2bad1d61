// Fused tensor-core (BF16) training pass of one network: kernel arguments and host entry
// points (the kernel is in ntbc_train_tc.cu).
#pragma once

#include "ntbc_internal.cuh"
#include "ntbc_kernels.cuh"
#include "ntbc_train_common.cuh"

namespace ntbc {

struct TrLayer {
    int K;                    // forward MMA K: input columns incl. the bias column, multiple of 16
    int N;                    // forward MMA N: 64 (hidden) or the padded output width
    int in, out;              // real sizes
    int img;                  // byte offset of the layer's [N][K] BF16 tile in the weight image
    long long w_off, b_off;   // parameter offsets of W [out][in] and b [out]
    int dw_col;               // TMEM column (within the group) of the weight-gradient accumulator
};

struct TrNet {
    int n_layers, K0, in_dim, out_dim, out_pad;
    TrLayer layer[NTBC_MAX_MLP_LAYERS];
    int img_bytes;            // hi tiles, then (lo_img > 0) the lo tiles at the same offsets + lo_img
    int lo_img;               // endpoint network: byte offset of the weights' lo parts (w - bf16(w),
                              // rounded to BF16; hi + lo carries ~16 bits), 0 for the colour network
    long long mlp_base;       // parameter offset of the network's first MLP weight
    int mlp_params;           // MLP parameters of the network (contiguous from mlp_base)
};

struct TrSmem {               // byte offsets: weight image at 0, then the groups
    int group_off, group_bytes;
    int x_off, a_off[3], d_off, bar_off;   // inside a group
    int x2_off;               // colour network: the second input tile (the helper gathers ahead);
                              // endpoint network: the lo parts of the input tile
    int alo_off;              // endpoint network: the lo parts of the hidden activations [128][64]
                              // (= d_off: the delta tile is dead during the forward)
    int stage_off;            // endpoint network: FP32 outputs and summed L_cd gradients, [128][out]
};

struct TrArgs {
    ModelView mv;
    TrNet net;
    TrSmem sl;
    GridSrc src;
    TexPtrs tp;
    const int32_t* ids;
    int B, tiles, groups, color;
    float T;
    float* grads;
    double* acc;
    int* err;
    const unsigned char* img;  // global BF16 weight image of this network
    float* partials;           // [grid * groups][mlp_params] weight-gradient partial sums
};

// layer table of one network (weight image offsets from 0)
TrNet train_tc_net_desc(const ModelView& mv, bool color);
// TMEM columns one warpgroup needs (data accumulator + every weight-gradient accumulator)
int train_tc_tmem_cols(const TrNet& n);
// BF16 weight image of the network from the FP32 master parameters (device img, img_bytes)
ntbc_status train_tc_images(const float* params, const TrNet& cnet, unsigned char* cimg, const TrNet& enet,
                            unsigned char* eimg, cudaStream_t s);
// rows of the partial-sum scratch a launch may use (one per warpgroup)
int train_tc_max_partial_rows();
// forward + loss + backward of B samples; adds the grid gradients into grads and the losses
// into the loss accumulators, and writes the MLP weight gradients as *rows partial rows of
// mlp_params floats into partials (scratch of max_rows rows), to be added by train_tc_reduce
ntbc_status train_tc_launch(const ModelView& mv, bool color, const TrNet& net, const unsigned char* img,
                            const GridSrc& src, const TexPtrs& tp, const int32_t* ids, int B, float T, float* grads,
                            double* acc, int* err, float* partials, int max_rows, int* rows, cudaStream_t s);
// grads[mlp_base + j] += the sum of each network's partial rows (both networks, one launch)
ntbc_status train_tc_reduce(const TrNet& cnet, const float* cpart, int crows, const TrNet& enet, const float* epart,
                            int erows, float* grads, cudaStream_t s);

}  // namespace ntbc
