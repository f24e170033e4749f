/*
 * lem_surrogate.h -- C ABI of the physics-informed sequence surrogate trained
 * on the solver's own probe series (arxiv 2510.22221: Results, "HPC and ML
 * framework", Fig. 2d-f; Methods "LEM Cell", Eq. discrete_lem; "ML Training
 * Implementation"; "Physics Loss", Eqs. ml_tra1-3 with the trapezoidal LLG
 * step of Eqs. llg_tra4-6).  Part of libfdtd_llg.so; errors use the FDTD_E_*
 * codes of fdtd_llg.h and fdtd_llg_last_error(NULL).
 *
 * Model.  An LEM cell (Eq. discrete_lem) with hidden width D maps
 * (y_{n-1}, z_{n-1}, u_n) to
 *   dt_n    = dt sigmoid(W1 y_{n-1} + V1 u_n + b1)
 *   dtbar_n = dt sigmoid(W2 y_{n-1} + V2 u_n + b2)
 *   z_n     = (1 - dt_n) z_{n-1} + dt_n tanh(Wz y_{n-1} + Vz u_n + bz)
 *   y_n     = (1 - dtbar_n) y_{n-1} + dtbar_n tanh(Wy z_n + Vy u_n + by)
 * The encoder stacks two cells (enc0 reads the input sample, enc1 reads
 * enc0's y_n) from zero states over t_in samples; the reconstruction of
 * sample n is Wo y_n of enc1.  The decoder stacks two cells with their own
 * weights (dec0, dec1), starts from the encoder's final (y, z) of the same
 * layer, reads 0 at its first step and then its previous output, and emits
 * Wo y_k of dec1 for t_out steps (one head Wo shared with the encoder, no
 * bias, as printed: o_n = W_y y_n).
 *
 * Losses (means over every element): L = MSE(recon, u) + MSE(out, target)
 * + lam L_phy.  Outputs are the two components of M/Ms transverse to the
 * bias (m = 2), in a right-handed frame (e1, e2, bias direction); the
 * component along the bias is taken as 1 (small-signal approximation, the
 * paper's "M_y ~ 0").  With m_k = (p_k, q_k, 1) and H_eff^k = h_k + h0 e3,
 * one trapezoidal step (Eqs. llg_tra4-6 with kappa = mu0 |gamma| dt_ML / 4,
 * H^{k+1}_eff in a, H^k_eff in b, normalised to |m_k|) gives F(m_k); the
 * residual F(m_k) - (p_{k+1}, q_{k+1}) for k = 0 .. t_out - 2 enters L_phy
 * as the mean of its squared components (Eqs. ml_tra1-3).
 *
 * Parameters: one flat FP32 vector of fdtd_llg_lem_param_count(d, m) values,
 * per cell c in the order enc0, enc1, dec0, dec1 (input width m_c = m for
 * enc0 and dec0, d for enc1 and dec1):
 *   W[4][d][d]    W1, W2, Wz, Wy (row i = output unit, column j = input unit)
 *   V[4][d][m_c]  V1, V2, Vz, Vy
 *   b[4][d]       b1, b2, bz, by
 * followed by Wo[m][d].
 *
 * Sequences (device FP32, sample-major, sequence next, component fastest):
 *   u[t_in][batch][m], target[t_out][batch][m], h[t_out][batch][3] (A/m, the
 *   frame components of the field at the predicted samples).
 *
 * Work space: fdtd_llg_lem_workspace_bytes() bytes of device memory, owned by
 * the caller, holding the saved activations of the last forward pass, the
 * outputs, their loss gradients, the gate gradients and the gradient
 * partials.  All pointers are device pointers unless stated; stream is a
 * cudaStream_t (NULL: the legacy default stream); every call is asynchronous
 * on that stream and reads nothing from the host after it returns.
 * Limits: d in {16, 32, 64}, 1 <= m <= 4 (m = 2 for lam != 0), batch >= 1,
 * t_in >= 1, t_out >= 1, t_in + t_out <= 65536.  Errors: FDTD_E_INVAL (a
 * limit, a NULL pointer), FDTD_E_CUDA (a launch failed).
 */
#ifndef LEM_SURROGATE_H
#define LEM_SURROGATE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int d;        /* hidden width D                                  */
    int m;        /* input and output width                          */
    int batch;    /* sequences per call                              */
    int t_in;     /* encoder samples                                 */
    int t_out;    /* decoder steps                                   */
    float dt;     /* the step dt of Eq. discrete_lem (> 0)           */
} fdtd_llg_lem_shape;

typedef struct {
    float lam;    /* weight of L_phy                                  */
    float kappa;  /* mu0 |gamma| dt_ML / 4, in m/A                     */
    float alpha;  /* Gilbert damping                                  */
    float h0;     /* bias field along the frame's third axis, A/m     */
} fdtd_llg_lem_physics;

/* Number of parameters for hidden width d and input width m (0 when out of
 * range). */
long long fdtd_llg_lem_param_count(int d, int m);

/* Work-space bytes for a shape (into *bytes).  Errors: FDTD_E_INVAL. */
int fdtd_llg_lem_workspace_bytes(const fdtd_llg_lem_shape *s, size_t *bytes);

/* Pointers into the work space: the reconstruction [t_in][batch][m] and the
 * prediction [t_out][batch][m] of the last forward pass (into *recon, *out),
 * the gradient of the last fdtd_llg_lem_loss/train_step call
 * [param_count] (into *grad) and its four losses as FP64 (total, L_rec,
 * L_pred, L_phy; into *loss).  Any output pointer may be NULL.  Errors:
 * FDTD_E_INVAL. */
int fdtd_llg_lem_views(const fdtd_llg_lem_shape *s, void *work, float **recon, float **out, float **grad,
                       double **loss);

/* Forward pass (encoder then decoder) of theta on u; results in the work
 * space (fdtd_llg_lem_views), activations saved for fdtd_llg_lem_backward.
 * Errors: FDTD_E_INVAL, FDTD_E_CUDA. */
int fdtd_llg_lem_forward(const fdtd_llg_lem_shape *s, const float *theta, const float *u, void *work, void *stream);

/* Losses of the last forward pass against u, target and h (see above), their
 * gradients with respect to the reconstruction and the prediction (kept in
 * the work space), and the four FP64 losses (fdtd_llg_lem_views).  h may be
 * NULL when lam = 0 (L_phy is then reported as 0).  Errors: FDTD_E_INVAL
 * (lam != 0 with m != 2 or without h), FDTD_E_CUDA. */
int fdtd_llg_lem_loss(const fdtd_llg_lem_shape *s, const fdtd_llg_lem_physics *p, const float *u,
                      const float *target, const float *h, void *work, void *stream);

/* Gradient of the total loss with respect to theta (back-propagation through
 * both stacks and the decoder's output feedback, then the sums of the gate
 * gradients against the saved activations in a fixed order: the result does
 * not depend on the launch configuration), into the work space's gradient.
 * Needs the forward pass and loss of the same theta and u.  Errors:
 * FDTD_E_INVAL, FDTD_E_CUDA. */
int fdtd_llg_lem_backward(const fdtd_llg_lem_shape *s, const float *theta, const float *u, void *work,
                          void *stream);

/* One Adam step (Kingma and Ba; beta1, beta2, eps; bias corrections for step
 * t >= 1) on n parameters: mom and vel are the caller's moment buffers
 * (zero before the first step).  Errors: FDTD_E_INVAL, FDTD_E_CUDA. */
int fdtd_llg_lem_adam(long long n, float *theta, const float *grad, float *mom, float *vel, float lr, float beta1,
                      float beta2, float eps, int t, void *stream);

/* One training step: forward, loss, backward and Adam (0.9, 0.999, 1e-8)
 * with learning rate lr at step t.  Errors: as the four calls. */
int fdtd_llg_lem_train_step(const fdtd_llg_lem_shape *s, const fdtd_llg_lem_physics *p, float *theta,
                            const float *u, const float *target, const float *h, float *mom, float *vel, float lr,
                            int t, void *work, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LEM_SURROGATE_H */
