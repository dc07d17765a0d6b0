/* spirit_gb_unet.h -- learned warm start for energy minimisation.
 *
 * The paper has no counterpart to anything in this header.  Its energy
 * minimiser (velocity projection, Appendix D) starts from a given spin
 * configuration; this network predicts, from a random initial configuration
 * and the Hamiltonian's parameters, a configuration near the one that
 * minimiser reaches, so that sp_minimise / sp_minimise_batch can finish the
 * relaxation from it.  The minimiser always finishes the job: the network's
 * output is only a starting point and is judged by the minimiser's energy and
 * max torque.
 *
 * Lattice and tensor layout.  The network works on an L x L periodic lattice
 * (the 2D hexagonal monolayer in its oblique cell coordinates): pixel (y, x)
 * is spin index x + L*y.  Activations are NHWC, BF16 (bit patterns passed as
 * uint16_t), pixel index p = (b*H + y)*W + x, channels innermost.  A 3x3
 * convolution is periodic in both directions:
 *     out[b,y,x,co] = bias[co] + sum_{t,ci} W[co][t][ci] * in[b,(y+dy)%H,(x+dx)%W,ci]
 * with tap t = 3*(dy+1) + (dx+1), dy, dx in {-1, 0, 1}, accumulated in FP32.
 *
 * Architecture (widths 32-64-128-256, every 3x3 convolution followed by ReLU):
 *   input   32 channels: n_x, n_y, n_z, f0, f1, f2, f3, then 25 zeros, where
 *           f = the caller's 4 per-system features, broadcast over the lattice
 *   e1a 32->32, e1b 32->32 (L)      pool 2x2 mean
 *   e2a 32->64, e2b 64->64 (L/2)    pool
 *   e3a 64->128, e3b 128->128 (L/4) pool
 *   b4a 128->256, b4b 256->256 (L/8)
 *   d3a [up(b4b) 256 | e3b 128] -> 128, d3b 128->128 (L/4)
 *   d2a [up(d3b) 128 | e2b 64]  -> 64,  d2b 64->64   (L/2)
 *   d1a [up(d2b) 64  | e1b 32]  -> 32,  d1b 32->32   (L)
 *   head y = Wh d1b + bh (1x1, 32->3, FP32), prediction m = y / |y|
 * up() is nearest-neighbour upsampling by 2 and [a | b] channel
 * concatenation; both are read on the fly, never stored.
 * Loss: mean over all pixels of 1 - m . m_target.
 *
 * Flat parameter vector (FP32; the order of sp_unet_layer's index): for each
 * of the 14 convolutions in the order above, W [Cout][9][Cin] then bias
 * [Cout]; then Wh [3][32], bh [3].  Layer e1a has Cin = 32 (its weights on
 * the 25 zero channels receive zero gradient).
 *
 * Spin records are 4 floats (x, y, z, pad), as for FP32 contexts.
 * Errors: SP_OK or a negative SP_ERR_* code (spirit_gb.h);
 * sp_unet_last_error gives the message.  Device pointers are the caller's,
 * never freed here; calls are asynchronous on `stream` unless stated.
 */
#ifndef SPIRIT_GB_UNET_H
#define SPIRIT_GB_UNET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define SP_UNET_LAYERS 14   /* 3x3 convolutions */
#define SP_UNET_IN_CH 32    /* padded input channels */
#define SP_UNET_FEATURES 4  /* per-system scalars broadcast as channels 3..6 */

typedef struct sp_unet sp_unet;

/* Parameter count of the flat vector. */
long long sp_unet_n_params(void);

/* Shape and flat offsets of convolution `layer` (0..13); layer 14 is the
 * head (cin 32, cout 3).  SP_ERR_ARG for another index. */
int sp_unet_layer(int layer, int *cout, int *cin, long long *w_offset, long long *b_offset);

/* Network for L x L lattices and batches of at most batch_max systems.
 * L must be a multiple of 8 and batch_max * (L/8)^2 a multiple of 128 for
 * every batch used (so every level's pixel count is a multiple of 128).
 * Allocates the weights, Adam moments and activation workspace (all device
 * memory of the network) on the current device.  Parameters start at zero;
 * set them with sp_unet_set_params. */
int sp_unet_create(sp_unet **out, int L, int batch_max);
void sp_unet_destroy(sp_unet *net);
const char *sp_unet_last_error(const sp_unet *net);

/* Copy the flat FP32 parameters from / to host memory (n = sp_unet_n_params).
 * set also zeroes the Adam moments and refreshes the BF16 weight copies.
 * Both synchronise the device. */
int sp_unet_set_params(sp_unet *net, const float *host, long long n);
int sp_unet_get_params(sp_unet *net, float *host, long long n);

/* Prediction for `batch` systems: spins_dev [batch][L*L] records, features_dev
 * [batch][4] floats, out_dev [batch][L*L] records (unit vectors, pad 0). */
int sp_unet_predict(sp_unet *net, const float *spins_dev, const float *features_dev, int batch, float *out_dev,
                    void *stream);

/* Loss and its gradient for one batch: target_dev [batch][L*L] records.
 * loss_dev (device, 1 double) receives the loss; the gradient (flat FP32,
 * n_params) is kept in the network for sp_unet_adam and, if grad_dev is not
 * NULL, copied there. */
int sp_unet_loss_grad(sp_unet *net, const float *spins_dev, const float *features_dev, const float *target_dev,
                      int batch, double *loss_dev, float *grad_dev, void *stream);

/* One Adam step (Kingma & Ba) with the gradient of the last
 * sp_unet_loss_grad; `step` counts from 1 (bias correction). */
int sp_unet_adam(sp_unet *net, double lr, double beta1, double beta2, double eps, int step, void *stream);

/* --- single kernels, for testing them one at a time ----------------------
 * Input of a convolution: channels [0, C0) from src0, [C0, C0+C1) from src1
 * (C1 = 0: no src1).  up0 != 0: src0 has H/2 x W/2 pixels and is upsampled
 * by 2 (nearest).  C0, C1, Cout multiples of 32; B*H*W a multiple of 128;
 * H, W even when up0. */

/* out = act(conv(in, W) + bias); act = ReLU if relu, identity otherwise;
 * bias may be NULL (zero); mask (same layout as out, may be NULL) zeroes
 * outputs whose mask value is not > 0 -- with the transposed weights of
 * sp_conv3x3_transpose this is the data gradient (ReLU derivative of the
 * layer's input as mask).  W [Cout][9][C0+C1] BF16, bias FP32. */
int sp_conv3x3_forward(const uint16_t *src0, int C0, int up0, const uint16_t *src1, int C1, const uint16_t *W,
                       const float *bias, int relu, const uint16_t *mask, int B, int H, int Wd, int Cout,
                       uint16_t *out, void *stream);

/* Wt[ci][8-t][co] = W[co][t][ci]: the weights of the data-gradient
 * convolution of a layer with W [Cout][9][Cin]. */
int sp_conv3x3_transpose(const uint16_t *W, int Cout, int Cin, uint16_t *Wt, void *stream);

/* Which kernel computes the 3x3 convolutions (forward and data gradient) of
 * this process: 3 (default) = tcgen05 on halo tiles for image rows of at
 * least 64 pixels (a CTA stages the input of a band of whole rows once per
 * 32-channel chunk and takes the nine taps as offsets into it) and kernel 1
 * for shorter rows or where the band does not fit; 1 = tcgen05 MMAs with
 * tensor-memory accumulators on a four-stage pipeline of one tap x 32
 * channels; 2 = the same with warp-specialised loads and MMA issue
 * (mbarrier pipeline); 0 = the mma.sync kernel.  SP_ERR_ARG for other
 * values.  Not thread-safe: set it before launching work. */
int sp_conv3x3_set_kernel(int tcgen05);
int sp_conv3x3_get_kernel(void);

/* SP_ERR_TIMEOUT if, since the last call, a convolution CTA gave up a bounded
 * wait on its tensor-core pipeline (its outputs were not written), else
 * SP_OK.  Synchronises the device and clears the flag. */
int sp_unet_device_error(void);

/* How many clock cycles a pipeline wait of the tcgen05 convolution (kernel
 * 1) and weight gradient (a stage waiting for the MMAs that read it) polls
 * before the CTA gives
 * up: it then stops loading and issuing, waits for the MMAs it issued (with
 * the default limit), frees its tensor memory, writes no output and sets the
 * flag sp_unet_device_error reports.  Default 2^32 (about two seconds); 0
 * makes every such wait give up at once.  SP_ERR_ARG if cycles < 0.  Process
 * wide and not thread-safe: set it before launching work.  The
 * warp-specialised kernel (2) keeps the default limit. */
int sp_conv3x3_set_wait_limit(long long cycles);

/* Workspace bytes sp_conv3x3_wgrad needs for this shape. */
long long sp_conv3x3_wgrad_workspace(int B, int H, int Wd, int Cin, int Cout);

/* Weight gradient dW[co][t][ci] = sum_p dz[p][co] * in_t[p][ci] (FP32) and,
 * if db is not NULL, db[co] = sum_p dz[p][co], with the input read as in
 * sp_conv3x3_forward.  Deterministic (fixed summation order).  With the
 * convolution kernel set to 1, 2 or 3 (sp_conv3x3_set_kernel) the products run
 * on tcgen05 MMAs (M = 128 tap-channel rows, N = output channels, K = the
 * pixels of one split, FP32 accumulators in tensor memory, splits added in a
 * fixed order; its pipeline waits obey sp_conv3x3_set_wait_limit); with 0
 * on mma.sync. */
int sp_conv3x3_wgrad(const uint16_t *src0, int C0, int up0, const uint16_t *src1, int C1, const uint16_t *dz, int B,
                     int H, int Wd, int Cout, float *dW, float *db, void *workspace, long long workspace_bytes,
                     void *stream);

#ifdef __cplusplus
}
#endif

#endif
