/* Learned proposal for global (re-)localisation: a PointNet-style network
 * maps a range scan to a Gaussian mixture over the sensor pose, from which
 * part of the particle set is seeded (the rest stays uniform).
 *
 * The paper initialises particles uniformly over the map (Sec. IV, the
 * initialisation and kidnapping experiments) and has no learned part; this is
 * an extension with its own sensor simulator, network, trainer and sampler.
 *
 * Network (FP32 parameters, FP32 arithmetic):
 *   x_p = scan point p / in_scale                        (P points x 3)
 *   h1 = relu(x W1 + b1)   3 -> 64      (shared over points)
 *   h2 = relu(h1 W2 + b2)  64 -> 128
 *   h3 = relu(h2 W3 + b3)  128 -> 256
 *   g  = max over points of h3          (256; ties -> smallest point index)
 *   h4 = relu(g W4 + b4)   256 -> 256
 *   o  = h4 W5 + b5        256 -> 416 = 32 components x (1 + 6 + 6)
 * o[c] = mixture logit a_c, o[32 + 6c + d] = mean m_cd, o[224 + 6c + d] = raw
 * log-std r_cd with log-std s_cd = 3 tanh(r_cd / 3). Parameters are one flat
 * float array in the order W1 b1 W2 b2 W3 b3 W4 b4 W5 b5, each W row-major
 * [in][out].
 *
 * Pose target of the mixture (6 values): y = ((x, y, z, yaw, pitch, roll) -
 * offset) / scale, angles the Z-Y-X Euler angles of the rotation; the yaw
 * difference y - m is wrapped into (-pi, pi] (scale[3] = 1, offset[3] = 0).
 * Loss of a sample: -log sum_c pi_c N(y; m_c, diag exp(2 s_c)), pi =
 * softmax(a); the batch loss is the mean over samples.
 *
 * All array pointers are DEVICE pointers; every call is enqueued on the
 * stream given at creation (mp_pn_sim_box_room takes its own). Return codes
 * are those of megaparticles.h; the message of a failure is
 * mp_last_error(NULL). */
#ifndef MP_PROPOSAL_H
#define MP_PROPOSAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MP_PN_OUT 416
#define MP_PN_COMPONENTS 32

typedef struct mp_pn mp_pn;

/* Box-room sensor simulator: ranges of rays from B poses along P sensor-frame
 * directions in a room [-half, half]^2 x [0, height] seen from inside, with
 * yawed boxes (boxes: n_boxes x 7 = centre x, centre y, base z, size x,
 * size y, size z, yaw). Output point = dir * (range + noise * N(0, 1)), the
 * normal draw from Philox-4x32-10 keyed by seed, counter (ray index, pose
 * index). poses: B x 7 (qx qy qz qw tx ty tz, sensor to world); dirs: P x 3
 * unit vectors; out: B x P x 3. A ray that hits nothing gives +inf. */
int mp_pn_sim_box_room(const float* boxes, int n_boxes, float half, float height, const float* poses, int64_t B,
                       const float* dirs, int P, float noise, uint64_t seed, float* out, void* cuda_stream);

/* Creates a network for scans of n_points points and batches of at most
 * max_batch scans, parameters initialised from seed (He-normal weights, zero
 * biases, last layer N(0, 0.01^2)). in_scale divides the scan coordinates;
 * scale[6], offset[6] define the pose target (above). */
int mp_pn_create(mp_pn** net, int n_points, int max_batch, float in_scale, const float scale[6],
                 const float offset[6], uint64_t seed, void* cuda_stream);
int mp_pn_destroy(mp_pn* net);
/* Number of parameters (floats of the flat array). */
int mp_pn_num_params(mp_pn* net, int64_t* n);
/* Copy the flat parameter array out of / into the network (device arrays). */
int mp_pn_get_params(mp_pn* net, float* out);
int mp_pn_set_params(mp_pn* net, const float* in);
/* Mixture outputs o (B x 416) of B scans (B x n_points x 3). */
int mp_pn_forward(mp_pn* net, const float* scans, int B, float* out);
/* Forward and backward pass: mean loss of the batch into *loss_dev (device
 * float) and the gradient of it w.r.t. the parameters into the network's
 * gradient buffer (copied to grad_out when it is not NULL). */
int mp_pn_loss_grad(mp_pn* net, const float* scans, const float* targets, int B, float* loss_dev, float* grad_out);
/* One Adam step (bias-corrected, step counter kept by the network) with the
 * gradient of the last mp_pn_loss_grad. */
int mp_pn_adam_step(mp_pn* net, float lr, float beta1, float beta2, float eps);
/* n poses (n x 7, qx qy qz qw tx ty tz) drawn from the mixture o (416 floats):
 * component by its softmax weight, then y = m + exp(s) * N(0, I), pose
 * values = y * scale + offset (yaw wrapped into (-pi, pi]), rotation from the
 * Z-Y-X Euler angles. Draws from Philox-4x32-10 keyed by seed, counter
 * (particle index). */
int mp_pn_sample(mp_pn* net, const float* mix, int64_t n, uint64_t seed, float* poses_out);

/* Arithmetic of the shared per-point layers (the network's only dense
 * contractions: 64 -> 128 and 128 -> 256 channels on every scan point).
 * MP_PREC_BF16 (the default when n_points is a multiple of 128): one fused
 * kernel on the tensor cores per forward pass -- layer 1 on the CUDA cores,
 * layers 2 and 3 as tcgen05 MMAs with BF16 weights and activations and FP32
 * accumulation, the max-pool in the same kernel; the FP32 parameters stay the
 * master copy (their BF16 image is refreshed at every update), and the
 * backward pass runs in FP32 on the activations the forward pass used.
 * MP_PREC_FP32: every layer on the CUDA cores in FP32. Returns MP_EINVAL for
 * another value, or for MP_PREC_BF16 when n_points is not a multiple of 128. */
int mp_pn_set_precision(mp_pn* net, int precision);
/* Waits for the network's stream; MP_ETIMEOUT if a bounded wait inside the
 * fused kernel gave up since the last call (its outputs are then invalid),
 * else MP_OK. */
int mp_pn_status(mp_pn* net);

#ifdef __cplusplus
}
#endif

#endif
