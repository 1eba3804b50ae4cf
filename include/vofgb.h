/*
 * vofgb.h -- C ABI of the GB300 (sm_103a) library for the hot path of the
 * one-fluid phase-change method of Malan, Malan, Zaleski & Rousseau,
 * "A Geometric VOF Method for Interface Resolved Phase Change and
 * Conservative Thermal Energy Advection" (arXiv:2001.03477):
 *   - PLIC reconstruction: MYC normal and plane constant (Sec. 3.2,
 *     Eq. plane_m),
 *   - Step 1, direction-split geometric VOF sweeps with divergence-free
 *     liquid velocity (Sec. 3.3.1, Eq. vof_step1_full; Weymouth-Yue split),
 *     the thermal energy fluxed in tandem with the same geometric fluxes
 *     (Sec. 3.4.1, Eq. disc_et_adv),
 *   - Step 2, the phase-change interface shift (Sec. 3.3.2,
 *     Eqs. vof_step2_full, Delta d, alpha^{n+1}) with the energy change
 *     Delta e = Delta c (C_pl - C_pg) T_Gamma (end of Sec. 3.4.1).
 *
 * Conventions
 *   - All array arguments are DEVICE pointers owned by the caller; the
 *     library allocates nothing on these calls.  Scalars are host values.
 *   - Cell arrays: double[nz][ny][nx], x fastest (no ghost cells; boundary
 *     conditions are applied by index mapping).
 *   - Face arrays of axis x: double[nz][ny][nx+1]; y: double[nz][ny+1][nx];
 *     z: double[nz+1][ny][nx]; face f lies between cells f-1 and f and
 *     holds the face-normal velocity (positive along +axis).  On a periodic
 *     axis face n is face 0 (the stored face-n value is not read).
 *   - PLIC plane of a mixed cell in its local unit cube (origin at the low
 *     corner): liquid is {x : m.x <= alpha}, m points from liquid into gas,
 *     |m_x| + |m_y| + |m_z| = 1.  Mixed cells: eps < c < 1 - eps.
 *   - Every call is asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream).  Host-side argument errors return VOF_EINVAL before
 *     anything is launched; launch failures return VOF_ECUDA.  Conditions
 *     detected inside kernels (a face CFL number above 1) set a sticky
 *     device status read by vof_get_device_status().
 *   - Out-of-place: input and output arrays of one call must not overlap.
 */
#ifndef VOFGB_H
#define VOFGB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define VOF_API __attribute__((visibility("default")))
#else
#define VOF_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VOF_OK = 0,
  VOF_EINVAL = 1,  /* bad argument (null pointer, size, aliasing) */
  VOF_ECUDA = 2,   /* a CUDA call failed; see vof_last_cuda_error() */
  VOF_ECFL = 3,    /* device status: |u| dt / h > 1 on some face */
  VOF_ESOLVE = 4,  /* an iterative solve (vof_velocity_extension,
                      vof_heat_diffusion) did not converge within max_iter,
                      or the extension's sub-domain has no free-flow face */
  VOF_EWAIT = 5    /* device status: a bounded wait of a tensor-core kernel
                      gave up (its results are not valid) */
} vof_status;

typedef struct {
  int nx, ny, nz;     /* interior cells per axis (>= 1; nx ny nz < 2^31) */
  int bc[3];          /* per axis x, y, z: 0 periodic, 1 zero-gradient */
  double h;           /* cell size (> 0) */
  double Cp_l, Cp_g;  /* volumetric heat capacities rho c_p of liquid, gas (> 0) */
  double T_sat;       /* interface temperature T_Gamma (Sec. 3.2: T_sat(p_sys)) */
  double eps_mixed;   /* mixed-cell threshold eps (Sec. 3.1: 1e-12) */
  int precision;      /* VOF_F64 (0): everything in FP64 (the paper's method).
                         VOF_F32_FLUX (1), the precision form: the sweeps'
                         MYC normals, PLIC slab volumes and WENO5 weights in
                         FP32; in FP64 the plane constants, the MYC decisions
                         wherever FP32 round-off could change them, the
                         empty/full test of a slab and its clamp to the
                         donor's liquid and gas, differences, updates, the
                         shift and all sums.  From the same input a sweep
                         agrees with VOF_F64 to ~4e-7 in c per cell; fluxes
                         telescope, so volume and energy are conserved to
                         FP64 round-off.  Any other value: VOF_EINVAL. */
  int scheme;         /* Step 1 sweeps (Sec. 3.3.1 names both):
                         VOF_SCHEME_WY (0): Weymouth-Yue, Eulerian donor slabs
                         and the dilatation term cc (a_r - a_l) with cc =
                         [c^n > 1/2] frozen at the step start (the default);
                         VOF_SCHEME_LE (1): Li's Lagrangian-explicit scheme
                         (CIAM): the velocity linear across a cell, the piece
                         of the donor that crosses a face is the preimage of
                         width |a| / J, J = 1 + (a_r - a_l) of the donor,
                         its liquid stretched by J is F, and the dilatation
                         term uses the cell's own c and Theta = (T C_pl) c +
                         (T C_pg)(1 - c) (no frozen state).  Any other value:
                         VOF_EINVAL. */
  int normal;         /* interface normal of the sweeps' reconstruction:
                         VOF_NORMAL_MYC (0): MYC (Sec. 3.2, the paper's method);
                         VOF_NORMAL_MLP (1): the learned normal of vof_mlp_*
                         (network parameters `mlp`) with MYC as its fallback,
                         for the mixed cells of each sweep (ghost donors
                         behind zero-gradient boundaries and the shift keep
                         MYC);
                         VOF_NORMAL_YOUNGS (2): Youngs' normal -grad c (the
                         1-2-1 weighted 3x3x3 gradient, L1-normalised), for the
                         same cells (a reference for shape-error comparisons).
                         Any other value: VOF_EINVAL. */
  const void* mlp;    /* VOF_NORMAL_MLP: device buffer of
                         vof_mlp_packed_bytes() bytes written by vof_mlp_pack
                         or vof_mlp_train_step (16-byte aligned); ignored
                         otherwise */
} vof_grid;

#define VOF_F64 0
#define VOF_F32_FLUX 1
#define VOF_SCHEME_WY 0
#define VOF_SCHEME_LE 1
#define VOF_NORMAL_MYC 0
#define VOF_NORMAL_MLP 1
#define VOF_NORMAL_YOUNGS 2

/* Number of doubles vof_step() writes to `sums`. */
#define VOF_NSUMS 6

/*
 * PLIC reconstruction (Sec. 3.2): for every mixed cell the MYC normal m
 * (Aulisa et al. 2007; centred-columns candidate kept unless its dominant
 * component exceeds the Youngs normal's) and the plane constant alpha with
 * V(m, alpha) = c (analytic inversion, Scardovelli & Zaleski 2000).
 *   c      [N]     volume fractions (read)
 *   m      [3][N]  SoA normal components (written; 0 for pure cells)
 *   alpha  [N]     plane constants (written; 0 for pure cells)
 *   mixed  [N]     1 for mixed cells, 0 otherwise (written)
 */
VOF_API vof_status vof_reconstruct(const vof_grid* g, const double* c, double* m, double* alpha, uint8_t* mixed,
                           void* stream);

/*
 * One direction sweep of Step 1 (Sec. 3.3.1) along x, y or z with the
 * energy fluxed in tandem (Sec. 3.4.1).  With a = u dt / h on each face, the
 * donor is the upwind cell; the face VOF flux F is the liquid volume of the
 * donor slab of width |a| next to the face (PLIC geometry for mixed donors,
 * c |a| for pure ones), the face temperature T_f is WENO5 of T = e / C_p(c)
 * (Shu 2009), and G = T_f (C_pl F + C_pg (a - F)) is the fluxed energy.
 * Each cell then takes (Weymouth-Yue dilatation terms)
 *   c' = c + (F_l - cc a_l) - (F_r - cc a_r),  clamped to [0, 1]
 *   e' = e + (G_l - Theta a_l) - (G_r - Theta a_r)
 * with cc = [c^n > 1/2] and Theta = C_p(cc) T^n frozen at the start of the
 * time step.
 *   c_in, e_in    [N] state before the sweep (e_in may be NULL: VOF only)
 *   c_out, e_out  [N] state after the sweep (must not overlap the inputs;
 *                 e_out ignored when e_in is NULL)
 *   u_face        face velocities of this axis (layout above)
 *   dt            time step; a = u dt / h
 *   state [N] (uint8, in/out) and theta [N] (double, in/out): the frozen
 *     step-start data.  state bit0 = the cell changed earlier in this step,
 *     bit1 = its cc; theta holds its Theta.  A cell with bit0 clear takes
 *     cc and Theta from its current (c, e).  Zero `state` before the first
 *     sweep of every time step; the sweep marks the cells it changes.
 *     state may be NULL only for a single sweep from a step start.
 *     The VOF-only form (e_in NULL) reads state but does not write it.
 *   flux_out      face array (nullable): receives F of every face
 *   diag          device double[1] (nullable): clipped volume is ADDED
 *                 (atomically; last bits depend on block order)
 *   workspace     device scratch of at least vof_sweep_workspace_bytes(g)
 *                 bytes, 256-byte aligned, caller-owned, not overlapping the
 *                 fields and not shared with concurrent calls
 */
VOF_API size_t vof_sweep_workspace_bytes(const vof_grid* g);
VOF_API vof_status vof_advect_sweep_x(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                                      double* e_out, const double* u_face, double dt, uint8_t* state,
                                      double* theta, double* flux_out, double* diag, void* workspace,
                                      size_t workspace_bytes, void* stream);
VOF_API vof_status vof_advect_sweep_y(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                                      double* e_out, const double* v_face, double dt, uint8_t* state,
                                      double* theta, double* flux_out, double* diag, void* workspace,
                                      size_t workspace_bytes, void* stream);
VOF_API vof_status vof_advect_sweep_z(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                                      double* e_out, const double* w_face, double dt, uint8_t* state,
                                      double* theta, double* flux_out, double* diag, void* workspace,
                                      size_t workspace_bytes, void* stream);

/*
 * Unfused energy sweep (Sec. 3.4.1, Eq. disc_et_adv): e' from the face VOF
 * fluxes F exported by a VOF-only sweep of the same axis.  T is taken from
 * (c_before, e_in).  Paired with vof_advect_sweep_*(e_in = NULL) it gives
 * the same e_out, state and theta bit for bit as the fused sweep.
 *   axis 0/1/2; c_before, c_after [N] VOF field before/after the sweep;
 *   e_in, e_out [N]; flux_F, u_face: face arrays of the axis;
 *   state/theta as for the sweep (updated for cells whose c or e changed;
 *   with VOF_SCHEME_LE the cell's own Theta is used and they are untouched).
 */
VOF_API vof_status energy_advect_consistent(const vof_grid* g, int axis, const double* c_before, const double* c_after,
                                    const double* e_in, double* e_out, const double* flux_F, const double* u_face,
                                    double dt, uint8_t* state, double* theta, void* stream);

/*
 * Step 2, the phase-change shift (Sec. 3.3.2): every mixed cell moves its
 * plane along its normal by dd cells (Delta d = -(mdot / rho_l) dt / h):
 * alpha* = alpha + |m|_2 dd capped to the cell, c = V(m, alpha*).  The
 * movement a cap cuts off continues in the neighbours the interface moves
 * into: a pure cell of the receding phase takes the largest volume swept in
 * it by the shifted plane of an adjacent mixed cell extended into it.  Every
 * changed cell gets e += Delta c (C_pl - C_pg) T_sat.
 *   c_in, e_in [N] -> c_out, e_out [N] (no overlap)
 *   dd [N] per-cell shift in cell units (nullable: dd_uniform everywhere)
 *   state [N] (nullable): zeroed for the next time step
 *   diag device double[5] (nullable), ADDED atomically:
 *     {sum Delta c, volume clamped away in receiving cells, sum Delta e,
 *      sum c_out, sum e_out}
 *   workspace: device scratch of at least vof_shift_workspace_bytes(g)
 *     bytes, 256-byte aligned, overlapping no other argument; owned by the
 *     caller, contents need not be initialised, busy until the launches on
 *     `stream` complete.
 * Returns VOF_EINVAL for a bad grid, null or overlapping arrays, a missing,
 * short or misaligned workspace; VOF_ECUDA if a launch fails.
 */
VOF_API size_t vof_shift_workspace_bytes(const vof_grid* g);
VOF_API vof_status vof_phase_change_shift(const vof_grid* g, const double* c_in, const double* e_in, double* c_out,
                                  double* e_out, const double* dd, double dd_uniform, uint8_t* state, double* diag,
                                  void* workspace, size_t workspace_bytes, void* stream);

/*
 * One full time step of the method (Sec. 3.1 steps 1-2: Step 1 the split
 * VOF sweeps of Sec. 3.3.1 with the thermal energy fluxed in tandem, Sec.
 * 3.4.1, Eq. disc_et_adv; Step 2 the interface shift of Sec. 3.3.2) on the
 * caller's stream: zero the frozen state, three
 * (g->scheme: Weymouth-Yue or Lagrangian-explicit)
 * sweeps in Strang-alternated order (x,y,z on even step_index, z,y,x on odd),
 * then the shift; c and e are updated in place (every sweep and the shift
 * read and write them directly; the workspace holds the frozen state, the
 * per-sweep lists, planes and face fluxes, and the partial sums).
 *   u, v, w        face velocities
 *   dd, dd_uniform as for vof_phase_change_shift
 *   sums           device double[VOF_NSUMS] (nullable), OVERWRITTEN with
 *                  {sum c, sum e (after the step), clipped volume of the
 *                   sweeps, shift sum Delta c, shift clamped volume,
 *                   shift sum Delta e}, reduced in a fixed order
 *                  (deterministic).
 *   workspace      device buffer of at least vof_step_workspace_bytes(g)
 *                  bytes, 256-byte aligned, caller-owned, not shared with
 *                  concurrent calls.
 */
VOF_API size_t vof_step_workspace_bytes(const vof_grid* g);
VOF_API vof_status vof_step(const vof_grid* g, double* c, double* e, const double* u, const double* v, const double* w,
                    double dt, long step_index, const double* dd, double dd_uniform, double* sums,
                    void* workspace, size_t workspace_bytes, void* stream);

/*
 * Many independent subdomains ("boxes") stepped together (the paper has no
 * counterpart: it steps one domain; this serves workloads of thousands of small, uneven domains such as
 * separate droplets).  Each box is one vof_step() on its own grid, arrays and
 * time step; the boxes are spread over `lanes` streams that run concurrently
 * and share nothing but the read-only inputs.
 *
 * The plan (host only, nothing launched): boxes in decreasing cell count (ties
 * by index) go one by one to the lane with the fewest cells so far (ties: the
 * lowest lane); a lane runs its boxes in that order, one after the other,
 * reusing one step workspace of the largest size its boxes need.
 *   lane_of_box    host int[nbox]: the lane of each box (written)
 *   lane_offset    host size_t[lanes]: byte offset of each lane's workspace
 *                  in the batch workspace (256-byte aligned; written)
 *   workspace_bytes  host: bytes the batch workspace needs (written)
 * vof_batched_workspace_bytes() returns the same total (0 for bad boxes).
 *
 * vof_batched_step(): records an event on `stream`, makes each lane stream
 * wait for it, queues each lane's boxes (vof_step with the box's own dt, dd,
 * dd_uniform and sums + VOF_NSUMS * box), then makes `stream` wait for every
 * lane.  Work queued on `stream` before the call is therefore complete before
 * any box starts, and work queued after it sees every box finished; under
 * stream capture of `stream` the lanes become parallel branches of the graph.
 *   boxes          host array of nbox vof_box; their c, e, u, v, w, dd device
 *                  arrays.  c and e of different boxes must not overlap each
 *                  other or the workspace; u, v, w, dd are read only and may
 *                  be shared between boxes of the same shape.
 *   step_index     the step's index (sweep order as vof_step)
 *   sums           device double[nbox][VOF_NSUMS] (nullable): each box's
 *                  vof_step sums
 *   lanes          >= 1; lane_streams: host array of `lanes` cudaStream_t
 *                  (NULL allowed when lanes == 1: the boxes run on `stream`)
 *   workspace      device, 256-byte aligned, >= the plan's workspace_bytes
 * nbox == 0 returns VOF_OK with nothing launched.  Every box is checked
 * before anything is launched (VOF_EINVAL for a bad grid, null array, dt < 0,
 * overlapping c/e arrays, a short or misaligned workspace); a CUDA failure
 * returns VOF_ECUDA after the lanes have been joined back into `stream`.
 * Events are created and destroyed inside the call; the lanes' streams must
 * not be used by other work while the call's work runs.
 */
typedef struct {
  vof_grid grid;
  double* c;                      /* device [N] */
  double* e;                      /* device [N] */
  const double* u, *v, *w;        /* device face arrays of the box */
  double dt;
  const double* dd;               /* device [N], nullable */
  double dd_uniform;
} vof_box;

VOF_API vof_status vof_batched_plan(const vof_box* boxes, int nbox, int lanes, int* lane_of_box, size_t* lane_offset,
                                    size_t* workspace_bytes);
VOF_API size_t vof_batched_workspace_bytes(const vof_box* boxes, int nbox, int lanes);
VOF_API vof_status vof_batched_step(const vof_box* boxes, int nbox, long step_index, double* sums, int lanes,
                                    void* const* lane_streams, void* workspace, size_t workspace_bytes,
                                    void* stream);

/*
 * The same batch as ONE launch per kernel of the time step (the grouped
 * form; the paper has no counterpart: it steps one domain per MPI rank): vof_group_create() carves every box's own step workspace out of
 * the caller's buffer and writes, once, every kernel's per-box arguments
 * and the CTA -> box maps of the grouped launches into the same buffer
 * (synchronising `stream`); vof_group_step() then runs a time step of every
 * box with ~22 launches on `stream` whatever the number of boxes: each CTA
 * finds its box and its block within that box's own launch shape, so every
 * box computes exactly what vof_step() computes on it (the same kernels, sum
 * rows and reductions: bit-identical results).  No host work per box; the
 * step can be captured in a CUDA graph.
 *   boxes         host array, as for vof_batched_step; all boxes share the
 *                 grid's precision and normal (VOF_NORMAL_MLP is not
 *                 grouped: VOF_EINVAL)
 *   sums          device double[nbox][VOF_NSUMS] or NULL: each box's step
 *                 sums, written by every vof_group_step()
 *   work_per_cta  cells per CTA of the grid-stride kernels (planes, faces,
 *                 shift lists; >= 32): the grouped launches' granularity
 *                 (results do not depend on it; the autotuner picks it)
 *   workspace     device, 256-byte aligned, vof_group_workspace_bytes()
 *                 bytes; it holds the boxes' workspaces and the tables while
 *                 the group lives.  Fields must not overlap it or each other.
 *   *group        host-side handle (launch sizes and table addresses);
 *                 vof_group_destroy() frees it (nothing on the device).
 * The boxes' arrays, dt, dd and sums are captured at creation: a later
 * change to them needs a new group.  VOF_EINVAL for a bad box, mixed
 * precision or normal, a small or misaligned workspace; VOF_ECUDA if the
 * table copy or a launch fails.
 */
typedef struct vof_group vof_group;
VOF_API size_t vof_group_workspace_bytes(const vof_box* boxes, int nbox, int work_per_cta);
VOF_API vof_status vof_group_create(const vof_box* boxes, int nbox, double* sums, int work_per_cta, void* workspace,
                                    size_t workspace_bytes, void* stream, vof_group** group);
VOF_API vof_status vof_group_step(vof_group* group, long step_index, void* stream);
VOF_API void vof_group_destroy(vof_group* group);

/*
 * Mass transfer rate from PLIC interface distances (Sec. 3.2, "Calculating
 * the mass transfer rate": Eqs. mdot_calc, grad_n_T, plane_m, cell_d,
 * dint_trans, the collinearity xi, normTgrad and the weights chi, gamma).
 * For each mixed cell (eps < c < 1 - eps): the MYC normal and plane constant
 * as in vof_reconstruct, in Hessian form n = m/|m|, d = alpha/|m| (n points
 * from liquid into gas).  Each pure cell within two cells of a mixed cell
 * (Chebyshev distance 1 or 2) takes the plane of its mixed neighbour of
 * largest collinearity xi = |n . dx| (dx from that neighbour's low corner
 * to the cell's centre; on ties the first in the order z, y, x of the
 * offsets, each increasing), the normal distance |d_Gamma| = |d - n . dx| h
 * and the temperature gradient along n, (T_Gamma - T)/|d_Gamma| in the
 * liquid (c > 1/2), (T - T_Gamma)/|d_Gamma| in the gas, with T = e / C_p(c)
 * and T_Gamma = g->T_sat; a cell on the plane (d_Gamma = 0) has none.  Each
 * mixed cell averages its pure neighbours' gradients per phase with weights
 * gamma = |n . dx| / |dx|^2 (dx the offset of the centres; a phase without
 * one contributes 0) and
 *     mdot = (k_g grad_g - k_l grad_l) / h_fg    (> 0: liquid turns to gas).
 * Offsets leaving the grid on a zero-gradient axis are not cells; periodic
 * axes wrap.
 *   c, e         device double[N] (cell layout), read only
 *   k_l, k_g     thermal conductivities (>= 0), h_fg latent heat (> 0)
 *   mdot         device double[N]: mdot at mixed cells, 0 elsewhere
 *   d_gamma      device double[N] or NULL: |d_Gamma| of each pure cell
 *                within two cells of a mixed cell, -1 elsewhere
 *   grad_n       device double[N] or NULL: that cell's gradient, 0 elsewhere
 *                (and where it has none)
 *   dd           device double[N] or NULL: dd_per_mdot * mdot at mixed cells,
 *                0 elsewhere -- with dd_per_mdot = -dt / (rho_l h), the shift
 *                Delta d of Step 2 (Eq. Delta d) for vof_phase_change_shift
 *   workspace    device buffer of vof_mass_transfer_workspace_bytes(g) bytes,
 *                256-byte aligned, caller-owned, not shared with concurrent
 *                calls
 * Outputs must not overlap each other, the inputs or the workspace.
 * VOF_EINVAL for a bad grid, null or overlapping arrays, a small or
 * misaligned workspace, h_fg <= 0 or a negative conductivity.
 */
VOF_API size_t vof_mass_transfer_workspace_bytes(const vof_grid* g);
VOF_API vof_status vof_mass_transfer(const vof_grid* g, const double* c, const double* e, double k_l, double k_g,
                                     double h_fg, double* mdot, double* d_gamma, double* grad_n, double dd_per_mdot,
                                     double* dd, void* workspace, size_t workspace_bytes, void* stream);
/* {mixed cells, pure cells with a mixed neighbour} of the last
 * vof_mass_transfer() run with this workspace (instrumentation; the paper
 * has no counterpart), copied to host memory after the work queued on
 * `stream` completes. */
VOF_API vof_status vof_mass_transfer_work_counts(const vof_grid* g, const void* workspace, int* counts,
                                                 void* stream);

/*
 * Velocity extension across the interface (Sec. 3.3.1: Eq. press_inv, the
 * correction u~ = -(dt/rho) grad p~ and u_l = u^{n+1} + u~).  Sub-domain:
 * the mixed cells and the pure gas cells (c <= eps) of the first two layers
 * around them, layers counted across cell faces.  Faces to pure liquid
 * cells (c >= 1 - eps) and zero-gradient walls are no-slip; faces to gas
 * cells beyond the second layer are free flow (p~ = 0 there); periodic axes
 * wrap.  In every sub-domain cell
 *   sum_faces beta_f (p~_Q - p~_P) = mdot (1/rho_g - 1/rho_l) A / h,
 *   beta_f = (dt / rho_f) / h^2, rho_f = rho_l c_f + rho_g (1 - c_f),
 *   c_f the mean of the two cells' c, A the PLIC plane area of a mixed
 *   cell in cell units (as in vof_reconstruct; gas cells: no source);
 * solved by preconditioned conjugate gradients until the residual falls to
 * tol times that of p~ = 0 (or max_iter iterations).  Then on every face
 * with a sub-domain cell on one side and no liquid cell or wall
 * u~ = -(dt / rho_f) (p~_R - p~_L) / h (p~ = 0 outside), 0 elsewhere.
 *   c, mdot      device double[N] (mdot read at mixed cells, e.g. from
 *                vof_mass_transfer)
 *   rho_l, rho_g densities (> 0); dt >= 0; tol > 0; max_iter >= 1
 *   u, v, w      device face arrays or all NULL: u~ is added (u_l = u + u~)
 *   ut, vt, wt   device face arrays or all NULL: u~ is written
 *   iterations, residual   host int / double or NULL: CG iterations and the
 *                final residual norm
 *   workspace    device buffer of vof_velocity_extension_workspace_bytes(g)
 *                bytes, 256-byte aligned, caller-owned
 * The call synchronises `stream` (the convergence test reads the residual).
 * VOF_EINVAL for bad arguments (also when neither u,v,w nor ut,vt,wt is
 * given); VOF_ESOLVE when the sub-domain has no free-flow face (nothing
 * fixes p~; outputs untouched) or CG did not converge (outputs written from
 * the last iterate).
 */
VOF_API size_t vof_velocity_extension_workspace_bytes(const vof_grid* g);
VOF_API vof_status vof_velocity_extension(const vof_grid* g, const double* c, const double* mdot, double rho_l,
                                          double rho_g, double dt, double tol, int max_iter, double* u, double* v,
                                          double* w, double* ut, double* vt, double* wt, int* iterations,
                                          double* residual, void* workspace, size_t workspace_bytes, void* stream);

/*
 * Implicit heat diffusion with the interface as a Dirichlet boundary
 * (Sec. 3.4.2: Eqs. T_diff_disc and mod_branchesT).  A node is liquid when
 * c >= 1/2, else gas; each phase diffuses with its own conductivity, and
 * T = T_Gamma = g->T_sat on the interface.  Along each axis the gradient
 * towards a same-phase neighbour is (T_nb - T)/h, towards the other phase
 * (T_Gamma - T)/theta, and the axis' second difference is divided by
 * (d_- + d_+)/2 (d = h or theta).  theta: the height function of the 7 cells
 * centred on the node along the axis when the column ends in pure cells of
 * the node's phase behind and the other phase beyond (H - 3.5 cells ahead of
 * a liquid node, 3.5 - H of a gas node), else the distance along the axis
 * to the PLIC plane of the pair's mixed cell (the node's own if mixed, else
 * the neighbour's), half a cell when both are pure or the plane is parallel
 * to the axis; capped to [1e-3 h, h].  Zero-gradient walls carry no flux,
 * unless wall_T gives the face a fixed temperature T_w: the node then sees
 * the wall half a cell away, gradient (T_w - T)/(h/2), d = h/2 (the heated
 * wall of the Stefan problem, Sec. 4.3).  Backward Euler with T = e/C_p(c),
 * solved by Jacobi sweeps (the system is strictly diagonally dominant)
 * until no T changes by more than tol in a sweep (or max_iter sweeps):
 *   VOF_CP_PHASE (the paper's phase-by-phase solve with constant properties
 *     in each phase): C_p,node (T' - T)/dt = k_p sum L(T'), C_p,node the
 *     heat capacity of the node's phase, and e' = e + C_p,node (T' - T);
 *   VOF_CP_MIXTURE: C_p(c) (T' - T)/dt = k_p sum L(T'), e' = C_p(c) T'.
 *   c            device double[N], read only
 *   e            device double[N], read and overwritten with e'
 *   k_l, k_g     conductivities (>= 0); dt > 0; tol > 0 (absolute, in T);
 *                max_iter >= 1
 *   heat_capacity  VOF_CP_PHASE or VOF_CP_MIXTURE
 *   wall_T       host double[6] or NULL: fixed temperatures of the faces
 *                x-, x+, y-, y+, z-, z+ (NaN: none); only on zero-gradient
 *                axes
 *   iterations, change   host int / double or NULL: sweeps made and the
 *                last sweep's largest change
 *   workspace    device buffer of vof_heat_diffusion_workspace_bytes(g)
 *                bytes, 256-byte aligned, caller-owned
 * The call synchronises `stream`.  VOF_EINVAL for bad arguments or
 * overlaps; VOF_ESOLVE when max_iter sweeps did not converge (e is written
 * from the last sweep).
 */
VOF_API size_t vof_heat_diffusion_workspace_bytes(const vof_grid* g);
#define VOF_CP_PHASE 0
#define VOF_CP_MIXTURE 1
VOF_API vof_status vof_heat_diffusion(const vof_grid* g, const double* c, double* e, double k_l, double k_g,
                                      double dt, double tol, int max_iter, int heat_capacity, const double* wall_T,
                                      int* iterations, double* change, void* workspace, size_t workspace_bytes,
                                      void* stream);

/*
 * Checkpoint and resume (host code; the paper has no counterpart): the
 * grid, the step index, the time and the fields c and e in one
 * little-endian file -- magic "VOFGBCK1", a fixed header, c[N], e[N], an
 * FNV-1a 64-bit checksum.  Save writes `path`.tmp and renames it into place.
 * Info reads the header into *g (and *step, *t when not NULL); load checks
 * magic, version, sizes (cells must equal the file's N) and checksum, then
 * copies c and e into the caller's host buffers.
 *   c, e           host double[N] (cell layout)
 * VOF_EINVAL for null arguments, an unreadable, truncated, foreign or
 * corrupted file, or a size mismatch.
 */
VOF_API vof_status vof_checkpoint_save(const char* path, const vof_grid* g, const double* c, const double* e,
                                       long step, double t);
VOF_API vof_status vof_checkpoint_info(const char* path, vof_grid* g, long* step, double* t);
VOF_API vof_status vof_checkpoint_load(const char* path, size_t cells, double* c, double* e);

/*
 * A time step that allocates nothing (the paper has no counterpart; this is
 * for callers that cannot allocate device memory when they step -- code in a
 * host callback or an error path where the allocator must not be entered,
 * embedders whose device memory is reserved up front by their own pool, small
 * tools without an allocator).  Same arguments and results as vof_step(),
 * minus the workspace: the scratch space is one fixed 40 MiB array that every
 * GPU loading the library keeps until the process exits.
 *   - grids above VOF_NOALLOC_MAX_CELLS cells, or whose step workspace
 *     (vof_step_workspace_bytes) exceeds the array -- only grids with fewer
 *     than 8 cells along some axis can -- return VOF_EINVAL, nothing
 *     launched;
 *   - all calls on a device share the array: calls whose kernels overlap on
 *     the GPU race (order them on one stream or synchronise in between);
 *   - the array keeps the previous call's contents; the step clears what must
 *     start at zero itself;
 *   - the first call on a device looks up the array's address with that
 *     device current; make it before any stream capture on the device.
 * vof_noalloc_scratch_bytes() returns the size of the array.
 */
#define VOF_NOALLOC_MAX_CELLS 262144L
VOF_API size_t vof_noalloc_scratch_bytes(void);
VOF_API vof_status vof_step_noalloc(const vof_grid* g, double* c, double* e, const double* u, const double* v,
                                    const double* w, double dt, long step_index, const double* dd, double dd_uniform,
                                    double* sums, void* stream);

/*
 * Work counts of the last vof_step() run with this workspace
 * (instrumentation; the paper has no counterpart): counts[VOF_NCOUNTS] =
 *   {mixed cells, faces evaluated} of the x, y and z sweeps (6 ints),
 *   {moving mixed cells by the analytic plane constant, by bisection,
 *    receivers settled} of the shift (3 ints),
 *   {learned normals replaced by MYC} of the x, y and z sweeps (3 ints; 0
 *    with VOF_NORMAL_MYC).
 * Copies them to host memory after the work queued on `stream` (the step's
 * stream) completes.  VOF_EINVAL for a bad grid or null pointers.
 */
#define VOF_NCOUNTS 12
VOF_API vof_status vof_step_work_counts(const vof_grid* g, const void* workspace, int* counts, void* stream);

/*
 * Per-launch timing (instrumentation; the paper has no counterpart).
 * vof_profile_begin(stream) records a start event on `stream`; until
 * vof_profile_end() every kernel or memset the library launches is followed
 * by an event on its stream.  vof_profile_end() waits for the last event,
 * writes up to max_entries launch durations in milliseconds (time from the
 * previous event, so each includes the gap before its launch) and the
 * launches' names (static strings owned by the library), and returns the
 * number of launches recorded (-1 if no profile was open or CUDA failed).
 * Profile one stream at a time.  VOF_EINVAL if a profile is already open.
 */
VOF_API vof_status vof_profile_begin(void* stream);
VOF_API int vof_profile_end(float* ms, const char** names, int max_entries);

/*
 * FP64 rate probe (instrumentation; the paper has no counterpart): `blocks`
 * CTAs of 256 threads, each thread running 8 independent chains of `iters`
 * dependent FP64 fused multiply-adds (op 0: 2 flops each) or adds (op 1:
 * 1 flop each); one double per thread is stored to out[blocks * 256]
 * (device).  The caller times it (CUDA events on `stream`): flops =
 * blocks * 256 * 8 * iters * (2 or 1).  VOF_EINVAL for a bad op, iters or
 * blocks < 1, or null out.
 */
VOF_API vof_status vof_fp64_probe(int op, long iters, int blocks, double* out, void* stream);

/*
 * Learned interface normal (the paper reconstructs with MYC, Sec. 3.2,
 * Eq. plane_m [Aulisa07]; the learned-normal form replaces that step): a
 * network 27 -> 64 -> 64 -> 3 with GELU (x Phi(x)) maps the 27 volume
 * fractions of a cell's 3x3x3 stencil (x fastest, inputs 2 c - 1) to the
 * normal direction y (liquid -> gas), m = y / |y|_1.  BF16 weights, FP32
 * accumulation on the tensor cores; activations enter the products as the
 * sum of three BF16 numbers (FP32-accurate).
 *
 * Parameters.  master: FP32 device vector of VOF_MLP_PARAMS values in the
 * order W1[64][27], b1[64], W2[64][64], b2[64], W3[3][64], b3[3] (W[out][in]).
 * packed: device buffer of vof_mlp_packed_bytes() bytes, 16-byte aligned,
 * the BF16 weight images the kernels load; vof_mlp_pack() writes it from
 * master (round to nearest even).
 *
 * vof_mlp_forward: y[n][3] (FP32) of the stencils X[n][27] (FP64 volume
 *   fractions), n >= 0.
 * vof_mlp_normals: the learned normal with the MYC fallback: the plane
 *   residual of a normal is the RMS over the 26 neighbours of (volume of the
 *   plane with that normal through the central cell's plane constant) - c,
 *   evaluated in FP32; the network's normal is kept when its residual is at
 *   most 1.25 x that of the MYC normal + 1e-3 (and |y|_1 > 0), else MYC
 *   (the precision form's MYC, decisions as in FP64).  m[n][3] (FP64,
 *   L1-normalised) and fallback[n] (nullable; 1 where MYC was taken).
 * Both: VOF_EINVAL for null pointers, n < 0, misaligned packed.
 */
#define VOF_MLP_PARAMS 6147
VOF_API size_t vof_mlp_packed_bytes(void);
VOF_API vof_status vof_mlp_pack(const float* master, void* packed, void* stream);
VOF_API vof_status vof_mlp_forward(const void* packed, const double* X, long n, float* y, void* stream);
VOF_API vof_status vof_mlp_normals(const void* packed, const double* X, long n, double* m, uint8_t* fallback,
                                   void* stream);

/*
 * One training step of the learned normal on the GPU (the paper has no
 * counterpart: the network stands in for the MYC normal of Sec. 3.2,
 * Eq. plane_m).  Forward, backward and Adam run in the library's kernels.
 * The loss is the batch mean of the squared distance between y / |y|_2 and
 * the label.  The batch holds `batch`
 * samples (a multiple of 128, 128 ... 65536) of the training set X[ntrain][27]
 * (FP64 fractions), N[ntrain][3] (FP64 unit normals): with idx == NULL
 * drawn with replacement, sample s of step `step` being
 * splitmix64(seed ^ splitmix64(step * 0x100000001B3 + s)) mod ntrain; else
 * idx[batch] (device, int64) gives them.  Gradients are taken with respect to
 * the BF16-rounded weights in `packed` (the values the forward pass uses)
 * and summed over 128-sample tiles in a fixed order (deterministic).  With
 * lr > 0: Adam (beta1 0.9, beta2 0.999, eps 1e-8, bias correction with
 * step >= 1) updates master, adam_m, adam_v (FP32, VOF_MLP_PARAMS each,
 * zero before step 1) and rewrites packed from the new master; with lr == 0
 * nothing but grad and loss is written.
 *   grad       device float[VOF_MLP_PARAMS] (nullable): the batch gradient
 *   loss       device float[1] (nullable): the batch-mean loss
 *   workspace  device, vof_mlp_train_workspace_bytes(batch) bytes, 256-byte
 *              aligned (per-tile partial sums)
 * VOF_EINVAL for a bad batch, ntrain < 1, null arrays, a short workspace.
 */
VOF_API size_t vof_mlp_train_workspace_bytes(int batch);
VOF_API vof_status vof_mlp_train_step(const double* X, const double* N, long ntrain, int batch,
                                      unsigned long long seed, long step, float lr, float* master, float* adam_m,
                                      float* adam_v, void* packed, float* grad, float* loss, const int64_t* idx,
                                      void* workspace, size_t workspace_bytes, void* stream);

/* Error reporting (the paper has no counterpart).
 *   vof_get_device_status()  the sticky device status (synchronises the
 *                            device): VOF_OK, VOF_ECFL or VOF_EWAIT;
 *                            reading clears it
 *   vof_status_string()      message for a status code (static string)
 *   vof_last_cuda_error()    the cudaError_t of the last call that returned
 *                            VOF_ECUDA */
VOF_API vof_status vof_get_device_status(void);
VOF_API const char* vof_status_string(int status);
VOF_API int vof_last_cuda_error(void);

#ifdef __cplusplus
}
#endif

#endif /* VOFGB_H */
