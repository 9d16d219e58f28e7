/*
 * kb.h — C ABI of the GB300 Keldysh loop-bubble library (libkb.so).
 *
 * The library evaluates the loop bubble of the single-impurity Anderson model in the
 * Keldysh formalism (KeldyshQFT paper, arXiv:2405.20996, Sec. II.D.1 "bubble_function"):
 *
 *     B_r(w, v, v') = c_r ∫ dv''/(2πi) Γ1(w, v, v'') Π_r(w, v'') Γ2(w, v'', v'),
 *
 * in the channels r = a, p, t (c_a = 1, c_p = 1/2 × 2 equal spin terms, c_t = −1 with the
 * up-up/up-down spin sum), for all 16 Keldysh components, with the propagator pair
 * Π = G G or Π-dot = G S + S G (Sec. II.C.5).  The v'' integral is the fixed composite
 * 5-point Gauss-Lobatto rule in the grid's auxiliary variable x (Sec. II.G.4–II.G.5);
 * vertices are the asymptotic classes K1, K2, K2', K3 per channel (Sec. II.C.1) read by
 * linear interpolation in x (Sec. II.G.7).  Loop parts of the multiloop flow (Sec. III.C:
 * one-loop Γ∘Π-dot∘Γ, left γ-dot∘Π∘Γ, right Γ∘Π∘γ-dot, central Γ∘Π∘(left part)) and the
 * parquet Bethe–Salpeter step (Sec. III.B) are bubbles of different vertex slots and
 * propagator pairs.
 *
 * Conventions: every vertex array holds the up-down spin component with the 16 Keldysh
 * components innermost, ordered (a1' a2' | a1 a2) lexicographically with 1 = classical,
 * 2 = quantum, component index c = 8 b1' + 4 b2' + 2 b1 + b2 (b = a − 1); complex numbers
 * are interleaved (re, im).  Class layouts (row-major):
 *     K1 [n1][16], K2 [n2w][n2v][16] (w, v), K2' [n2w][n2v][16] (w, v'),
 *     K3 [n3w][n3v][n3v][16] (w, v, v').
 * Grids: N points v_i = A tan(π x_i / 2), x_i = −1 + 2(i+1)/(N+1), the same map for every
 * axis; classes read as 0 at x = ±1 (v = ±∞).
 *
 * Memory: all vertex pointers are DEVICE pointers owned by the caller, who keeps them
 * alive and unmodified until the work of the next kb_bubble on the given stream is done.
 * The library owns its context, its device tables and its workspace.
 * Errors: every call returns a kb_status and never aborts; kb_last_error() describes the
 * last failure.  Calls are asynchronous on the given cudaStream_t (NULL = legacy default
 * stream).  There is no CPU fallback: without a CUDA device kb_create fails.
 */
#ifndef KB_H
#define KB_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kb_ctx kb_ctx;

typedef enum {
    KB_OK = 0,
    KB_ERR_ARG = 1,          /* invalid argument (range, null, size mismatch) */
    KB_ERR_STATE = 2,        /* call order violated (e.g. bubble before set_grids) */
    KB_ERR_CUDA = 3,         /* a CUDA runtime call failed; see kb_last_error */
    KB_ERR_OOM = 4,          /* device allocation failed */
    KB_ERR_TIMEOUT = 5,      /* a bounded device-side wait gave up */
    KB_ERR_UNSUPPORTED = 6,  /* combination not built (e.g. precision on this device) */
    KB_ERR_TOO_LARGE = 7     /* problem does not fit the fixed scratch of kb_bubble_fp64_noalloc */
} kb_status;

enum { KB_CH_A = 0, KB_CH_P = 1, KB_CH_T = 2 };
enum { KB_K1 = 0, KB_K2 = 1, KB_K2P = 2, KB_K3 = 3 };
#define KB_MASK_ALL 0xFu
enum { KB_PI_GG = 0, KB_PI_GS_SG = 1 };           /* Π = G G,  Π-dot = G S + S G */
enum { KB_REG_DELTA = 0, KB_REG_U = 1, KB_REG_T = 2, KB_REG_NONE = 3 };   /* flow schemes (kb_set_regulator) */
enum { KB_DT_C128 = 0, KB_DT_C64 = 1 };           /* complex double / complex float */
enum { KB_PREC_FP64 = 0, KB_PREC_MIXED = 1 };     /* plain FP64 / FP32 gather + 3xTF32 tensor-core contraction */
#define KB_MAX_SLOTS 16

/* Frequency grids of the vertex classes and the quadrature (Sec. II.G.4, II.G.5).
 * nq must be 4P + 1 (P panels of the composite 5-point Gauss-Lobatto rule). */
typedef struct {
    int n1;          /* K1 bosonic points */
    int n2w, n2v;    /* K2 / K2' bosonic and fermionic points */
    int n3w, n3v;    /* K3 bosonic and fermionic points */
    int nq;          /* quadrature nodes on x in [-1, 1], endpoints included */
    double A;        /* grid scale (v = A tan(pi x / 2)) */
} kb_grid_desc;

/* Create a context on CUDA device `device`.  Fails with KB_ERR_CUDA if there is none. */
kb_status kb_create(kb_ctx **ctx, int device);
kb_status kb_destroy(kb_ctx *ctx);

/* Set the class grids and the quadrature (Sec. II.G.4–5).  Invalidates nothing owned by
 * the caller; must precede kb_bubble. */
kb_status kb_set_grids(kb_ctx *ctx, const kb_grid_desc *g);

/* Model (Sec. I.A, III.A.1): flat hybridisation Δ, temperature T (T = 0 allowed), and the
 * effective level eps (0 for the symmetric model with the Hartree shift absorbed).
 * G^R(v) = 1/(v − eps + iΔ − Σ^R(v)), G^K = G^R [Σ^K − 2iΔ tanh(v/2T)] G^A, and the
 * hybridisation-flow single-scale propagator S = ∂G/∂Δ at fixed Σ (Sec. III.C.2). */
kb_status kb_set_model(kb_ctx *ctx, double Delta, double T, double eps);

/* Optional dynamic self-energy (Sec. II.C.2): n_sig points on a tan grid of scale A_sig,
 * interleaved complex double HOST arrays (copied); Σ reads 0 at x = ±1.  sigR == NULL
 * resets Σ = 0.  sigK may be NULL (Σ^K = 0). */
kb_status kb_set_self_energy(kb_ctx *ctx, int n_sig, double A_sig, const double *sigR, const double *sigK);

/* Flow scheme (Sec. III.C.2) of the single-scale propagator S = dG/dΛ at fixed Σ used by
 * KB_PI_GS_SG (default KB_REG_DELTA):
 *   KB_REG_DELTA  hybridisation flow, Λ = Δ: S^R = -i (G^R)^2;
 *   KB_REG_U      interaction flow at Λ = lambda > 0: the propagator itself becomes
 *                 G^R = λ / (v - eps + i Δ - λ Σ^R), G^K = G^R [Σ^K - 2 i Δ tanh(v/2T) / λ] G^A
 *                 (so Π = G G scales by λ^2 at Σ = 0), and S^R = (v - eps + i Δ) / (v - eps +
 *                 i Δ - λ Σ^R)^2; `lambda` is ignored by the other schemes;
 *   KB_REG_T      temperature flow, Λ = T (T > 0): S^R = 0, S^K = G^R (i Δ v / (T^2
 *                 cosh^2(v/2T))) G^A;
 *   KB_REG_NONE   no flow parameter: S = 0, so that with the Katanin tables of
 *                 kb_set_self_energy_derivative KB_PI_GS_SG uses G dΣ G alone — the change
 *                 of G (Dyson equation) along a change dΣ of the self-energy, e.g. for the
 *                 Jacobian of a self-consistent Σ.
 * S^K is always dG^K/dΛ of the general Keldysh component.  At x = ±1 the tail uses the
 * limits v G -> λ [[0,1],[1,0]] and v S -> [[0,1],[1,0]] (interaction flow) or 0. */
kb_status kb_set_regulator(kb_ctx *ctx, int kind, double lambda);

/* Katanin substitution (Sec. III.C.2: the differentiated propagator G-dot = S + G Σ-dot G):
 * n_dsig values of dΣ^R/dΛ (and dΣ^K/dΛ, may be NULL) on the tan grid of scale A_dsig,
 * interleaved complex double HOST arrays (copied), read linearly in x with zero at
 * x = ±1.  KB_PI_GS_SG then uses G-dot in place of S.  dsigR == NULL switches it off. */
kb_status kb_set_self_energy_derivative(kb_ctx *ctx, int n_dsig, double A_dsig, const double *dsigR,
                                        const double *dsigK);

/* Tabulated lines (the propagator pair of the bubble, Sec. II.C.5, and the line of the loop,
 * Sec. II.D.2, built from given propagators instead of from the model and Σ, Sec. II.C.2):
 * which = KB_PROP_G: G^R and G^K; which = KB_PROP_S: the single-scale propagator S^R and S^K.
 * n points on the tan grid v_i = A_tab tan(π x_i / 2), x_i = -1 + 2(i+1)/(n+1), interleaved
 * complex double HOST arrays (copied before the call returns), read linearly in x with zero at
 * x = ±1; the advanced part is the conjugate of the retarded one and the quantum-quantum
 * component is 0.  tabR == NULL removes that table (back to the model's line); tabK may be
 * NULL (zero Keldysh part).  A tabulated line replaces the model and the Σ tables for that
 * line; the Katanin tables still add G dΣ G to S, with the tabulated G.  While G is tabulated,
 * the S line (KB_PI_GS_SG, kb_loop line 1) needs an S table (KB_ERR_STATE otherwise), and the
 * G^R gradient of kb_bubble_vjp is not available with either table (KB_ERR_UNSUPPORTED).  The
 * endpoint terms at x = ±1 keep the asymptotics of the model and the flow scheme
 * (v G^R -> λ, v G^K -> 0, v S per scheme), so the tables should hold lines with those
 * asymptotics, e.g. of a self-energy that vanishes as |v| -> ∞.  Errors: KB_ERR_ARG (which,
 * n < 1, A_tab <= 0, a non-finite entry), KB_ERR_CUDA (device copy).  Step graphs captured
 * before the call refuse to launch afterwards. */
#define KB_PROP_G 0
#define KB_PROP_S 1
kb_status kb_set_propagator_table(kb_ctx *ctx, int which, int n, double A_tab, const double *tabR,
                                  const double *tabK);

/* Vertex slot `slot` (0 .. KB_MAX_SLOTS-1): the bare part R = Γ0 of the parquet
 * approximation (Sec. I.B: -U/2 on components with an odd number of quantum indices)
 * when has_R != 0, and no classes.  Classes are attached with kb_set_vertex_class. */
kb_status kb_set_vertex(kb_ctx *ctx, int slot, int has_R, double U);

/* Channels that are part of the vertex in slot `slot` (bit 1 << KB_CH_x; default all
 * three after kb_set_vertex).  The up-up spin component needed by the t channel is built
 * channel by channel (SU(2) + crossing, Sec. II.G.3): gamma_c^uu(1'2'|12) =
 * gamma_c^ud(1'2'|12) - gamma_sigma(c)^ud(1'2'|21), sigma: a <-> t, p -> p, so the data of
 * an excluded channel is still read as the crossing partner of an included one.  Use it
 * for the multiloop corrections, whose vertex is the sum over the channels other than r
 * (Sec. III.C). */
kb_status kb_set_vertex_channels(kb_ctx *ctx, int slot, unsigned mask);

/* Declare that the vertex in slot `slot` obeys complex conjugation and crossing symmetry
 * (Sec. II.G.3; in channel variables, conjugation: a,p (w,v,v') -> (w,v',v), t -> (-w,v,v')
 * with Keldysh (a1'a2'|a1a2) -> (a1a2|a1'a2'), conj and sign (-1)^(1+sum a); crossing:
 * a,t (w,v,v') -> (-w,v',v), p -> (w,-v,-v') with (a1'a2'|a1a2) -> (a2'a1'|a2a1)).  A bubble
 * of such a vertex with itself (slot_left == slot_right, beta == 0) then computes only the
 * independent part of the output (K2 for w >= 0 in a and t, for v >= 0 in p; K1 and K3 for
 * w >= 0 in a and t; the right K3 tile from the left one) and fills the rest by the same
 * symmetries.  The caller vouches for the symmetry; nothing checks it. */
kb_status kb_set_vertex_symmetric(kb_ctx *ctx, int slot, int symmetric);

/* Attach class `cls` of channel `channel` of slot `slot`: DEVICE pointer in the layout
 * above, dtype KB_DT_C128 or KB_DT_C64 (all classes of a slot need not share a dtype).
 * ptr == NULL detaches (the class reads as zero). */
kb_status kb_set_vertex_class(kb_ctx *ctx, int slot, int channel, int cls, void *dev_ptr, int dtype);

/* The bubble of channel `channel` with Γ1 = slot_left, Γ2 = slot_right and propagator pair
 * pi_kind, written into the classes (class_mask bits 1 << KB_K1 .. 1 << KB_K3) of channel
 * `channel` of slot out_slot:  out ← alpha · B + beta · out  (the paper adds, Sec. II.D.1;
 * beta = 1 reproduces that).  Γ1 is the vertex carrying the external v (for t: the vertex on
 * the external legs 1', 1).  precision: KB_PREC_FP64 (plain, every step in FP64) or
 * KB_PREC_MIXED (FP32 gather, 3xTF32 tensor-core contraction with FP32 accumulation;
 * propagators, Π and the tail in FP64; its input classes must be complex64 with 16-byte
 * aligned pointers, as every cudaMalloc or PyTorch allocation is).  The out slot's classes
 * must be attached and must not alias the inputs. */
kb_status kb_bubble(kb_ctx *ctx, int channel, int slot_left, int slot_right, int out_slot, int pi_kind,
                    unsigned class_mask, double alpha, double beta, int precision, void *stream);

/* The t-channel bubble of a vertex with itself in its SU(2) form (the symmetry reduction of
 * the spin sums, Sec. II.G.3, of the t bubble drawn in Sec. III.B): with Γ^d = Γ_uu + Γ_ud the
 * density combination and X the exchange of legs 1 and 2, the magnetic combination is
 * Γ_uu − Γ_ud = −X[Γ_ud], and exchanging legs 1 and 2 turns the t bubble into the a bubble,
 * so   B_t(Γ, Γ) = ½ (−Γ^d Π_t Γ^d) + ½ X[B_a(Γ, Γ)],
 * where X[B_a](w, v, v') = B_a(−w, v, v') with the Keldysh indices a1, a2 exchanged.  The
 * density contraction has one spin record per side, half the quadrature length of the two
 * spin terms kb_bubble contracts.  Two calls:
 *   kb_bubble_t_su2: out ← α B_t for K1, K2, K2' (as kb_bubble with β = 0, mixed precision)
 *     and, for K3, α/2 times the density contraction at the independent points (w ≥ 0,
 *     v ≤ v'); slot: a slot declared symmetric (kb_set_vertex_symmetric) with its bare part
 *     or channel t; out_slot: channel t classes attached (KB_ERR_STATE otherwise);
 *   kb_t_su2_finish: K3 of channel t of out_slot += α/2 X[a_k3] at those points, then its
 *     other points as the t channel's symmetry images; a_k3: DEVICE array, the K3 class
 *     [n3w][n3v][n3v][16] (c64 or c128, a_dtype) of B_a(Γ, Γ) with α = 1, β = 0, the same
 *     vertex, propagator pair, grids and model — e.g. another context's output, which the
 *     caller orders before this call (same stream, an event, or a step graph's
 *     KB_OP_T_SU2_FINISH entry).
 * Precision: mixed only (the K3 density contraction on tcgen05); asynchronous on `stream`. */
kb_status kb_bubble_t_su2(kb_ctx *ctx, int slot, int out_slot, int pi_kind, unsigned class_mask, double alpha,
                          void *stream);
kb_status kb_t_su2_finish(kb_ctx *ctx, int out_slot, const void *a_k3, int a_dtype, double alpha, void *stream);

/* Vector-jacobian product (adjoint) of kb_bubble (the differentiation pattern of the
 * method: gradients of a scalar loss through B_r, e.g. for Newton-Krylov solves of the
 * parquet equations, Sec. III.B).
 *
 * Convention: gradients of a real loss L on the real embedding (real and imaginary parts
 * as independent reals), bar(z) = dL/dRe z + i dL/dIm z, PyTorch's convention for complex
 * tensors.  The classes (class_mask) of channel `channel` of slot gout_slot hold
 * bar(out) for out = alpha B_r(Γ_left, Γ_right; Π) (+ beta out, which does not involve the
 * vertices).  The call ACCUMULATES:
 *   grad_left_slot  (or -1): classes += alpha J_left^H  bar(out), J_left = dB/d(stored
 *                    classes of slot_left) — every attached class of every channel of the
 *                    gradient slot receives its share (interpolation corners, channel
 *                    conversion and the up-up crossing partners of the forward);
 *   grad_right_slot (or -1): the same for slot_right (the two may be the same slot, then
 *                    both contributions add, as for B(Γ, Γ));
 *   grad_GR_K1/K2/K3 (device, complex128, or NULL): the gradient with respect to G^R at the
 *                    propagator samples of the output classes on that bosonic grid:
 *                    [w][node][side], w on the K1 (n1), K2 (n2w; K2 and K2' add) or K3
 *                    (n3w) grid, side 0 the propagator at v''+w/2 (a, t) or w/2+v'' (p),
 *                    side 1 at v''-w/2 or w/2-v''; G^A = (G^R)* and G^K = tanh(v/2T)(G^R -
 *                    G^A) are taken as functions of G^R (equilibrium FDR, Sec. II.C.4).
 *                    Needs pi_kind KB_PI_GG and no self-energy table (else
 *                    KB_ERR_UNSUPPORTED; also with a dΣ/dΛ table); the tail nodes (v'' = ±inf) carry no G dependence.
 * Gradient classes must be complex128 and must not alias any input.  The bare part
 * R = Γ0 is a fixed parameter (no gradient).  precision: KB_PREC_FP64 (every step in FP64)
 * or KB_PREC_MIXED (the input vertices complex64 and 16-byte aligned, else KB_ERR_ARG: their
 * records evaluated as the mixed forward evaluates them, FP32 tiles and GEMMs, while the
 * scatter into the complex128 gradient classes and the Π gradient accumulate in FP64; the
 * Π table and the pull-back to G^R are FP64); any other value is KB_ERR_ARG. */
kb_status kb_bubble_vjp(kb_ctx *ctx, int channel, int slot_left, int slot_right, int gout_slot, int pi_kind,
                        unsigned class_mask, double alpha, int grad_left_slot, int grad_right_slot,
                        void *grad_GR_K1, void *grad_GR_K2, void *grad_GR_K3, int precision, void *stream);

/* ---------------------------------------------------------------------------------------
 * Step graphs (batching): a list of bubbles of one or several contexts — several
 * parameter points, each with its own grids, model and vertices, the loop parts of a
 * multiloop step (Sec. III.C: one-loop, left, right and central parts are bubbles with
 * different slots and propagator pairs) and the three channels — captured once into a
 * CUDA graph and replayed with one launch per step.
 *
 * kb_graph_create sizes every context's workspace for its bubbles, does the one-time
 * device setup, and captures the bubbles (each as kb_bubble would run it) without running
 * them.  Bubbles of the same context run in list order; bubbles of different contexts
 * are independent branches of the graph and may overlap on the GPU, so they must not
 * write an array another branch reads or writes.  The graph holds the device pointers
 * and parameters in force at creation: later kb_set_* calls do not change it; the caller
 * keeps the contexts and every attached array alive until kb_graph_destroy.  All contexts
 * must be on one device.  On failure nothing is kept and the message is in
 * kb_last_error of the context of the failing (or the first) descriptor.
 * kb_graph_launch enqueues one replay on `stream` (asynchronous, like kb_bubble); it returns
 * KB_ERR_STATE without launching once a context of the graph has replaced device memory the
 * captured kernels address (its workspace grew for a larger bubble, kb_set_grids,
 * kb_set_self_energy(_derivative), or a record cache was freed or re-allocated) — create
 * the graph again then.  kb_graph_kernel_count gives the kernels one replay runs.
 * --------------------------------------------------------------------------------------- */
typedef struct kb_graph kb_graph;

/* Entry kinds of a step graph (kb_bubble_desc.op; zero-initialise the descriptor):
 *   KB_OP_BUBBLE  kb_bubble(ctx, channel, slot_left, slot_right, out_slot, pi_kind,
 *                 class_mask, alpha, beta, precision);
 *   KB_OP_ADD     kb_vertex_add(ctx, channel, slot_left, out_slot, class_mask, alpha);
 *   KB_OP_JOIN    every later entry, on every branch, waits for every earlier entry of
 *                 every branch (ctx may be NULL; the other fields are ignored) — the
 *                 point where the next loop order of a multiloop step reads the
 *                 derivatives of all channels of the previous one;
 *   KB_OP_CACHE   kb_vertex_cache(ctx, slot_left, channel, class_mask = sides): the record
 *                 cache is allocated at graph creation and rebuilt at every replay;
 *   KB_OP_IMAGE   kb_vertex_image(ctx, channel, slot_left, out_slot, class_mask);
 *   KB_OP_T_SU2   kb_bubble_t_su2(ctx, slot_left, out_slot, pi_kind, class_mask, alpha);
 *   KB_OP_T_SU2_FINISH  kb_t_su2_finish(ctx, out_slot, K3 of channel a of slot slot2 of
 *                 context ctx2, alpha), after every earlier entry of ctx2's branch (ctx2
 *                 must have entries in the graph; ctx's branch waits for them there). */
enum { KB_OP_BUBBLE = 0, KB_OP_ADD = 1, KB_OP_JOIN = 2, KB_OP_CACHE = 3, KB_OP_IMAGE = 4, KB_OP_T_SU2 = 5,
       KB_OP_T_SU2_FINISH = 6 };

typedef struct {
    kb_ctx *ctx;
    int channel, slot_left, slot_right, out_slot, pi_kind;
    unsigned class_mask;
    double alpha, beta;
    int precision;
    int op;
    kb_ctx *ctx2;                   /* KB_OP_T_SU2_FINISH: the context and slot of B_a */
    int slot2;
} kb_bubble_desc;

kb_status kb_graph_create(kb_graph **graph, const kb_bubble_desc *bubbles, int n);
kb_status kb_graph_launch(kb_graph *graph, void *stream);
kb_status kb_graph_kernel_count(kb_graph *graph, unsigned long long *count);
kb_status kb_graph_destroy(kb_graph *graph);

/* Slot arithmetic: the classes (class_mask) of channel `channel` of slot_dst
 * += alpha * those of slot_src, elementwise in the destination's precision (c64 or c128;
 * the source may have either).  Absent source classes read zero; a destination class
 * must be attached where the source has one, and must not be the same array.  Used
 * between the bubbles of a multiloop step (Sec. III.C: the l-loop derivative of channel r
 * is the sum of its left, central and right parts).  Asynchronous on `stream`. */
kb_status kb_vertex_add(kb_ctx *ctx, int channel, int slot_src, int slot_dst, unsigned class_mask, double alpha,
                        void *stream);

/* Symmetry image (Sec. II.G.3): the classes (class_mask, of the destination) of channel
 * `channel` of slot_dst are overwritten with the image of those of slot_src — conjugation
 * in a and p (w, v, v') -> (w, v', v), conjugation after crossing in t (the same w, v <-> v'),
 * with the Keldysh permutations, complex conjugation and sign (-1)^(1+Σa); destination K2
 * comes from source K2' and vice versa.  For conjugation- and crossing-symmetric Γ and X the
 * right part B_r(Γ, X) is the image of the left part B_r(X, Γ), so a multiloop order whose
 * input is symmetric needs one of the two bubbles.  Source and destination classes must be
 * attached, of one dtype and distinct.  Asynchronous on `stream`. */
kb_status kb_vertex_image(kb_ctx *ctx, int channel, int slot_src, int slot_dst, unsigned class_mask, void *stream);

/* Record cache of a vertex slot (mixed precision; Sec. II.C.1 class split), for the
 * bubbles of channel `channel`.  Sides (bits of `sides`):
 *   1  the part of the vertex that the K2 contraction gathers at every node as the left
 *      vertex — the other channels' classes at the converted frequencies, FP32, 16
 *      components (two spin records for t) — at every (w, v) of the K2 grids and interior
 *      node: n2w * n2v * (nq - 2, rounded up to a multiple of 32) * 128 bytes (twice for t);
 *   2  the same as the right vertex of the K2' contraction (records at (w, v''_j, v'));
 *   4  the K3 left tile of every bosonic frequency (TF32 hi/lo planes as the tensor-core
 *      contraction reads them): n3w * 4 * (4 n3v) * (4 nq) * 4 bytes (twice for t);
 *   8  the K3 right tile with Π = G G folded in (used by bubbles with KB_PI_GG).
 * Allocated by the library.  Later
 * mixed-precision bubbles of `channel` that have this slot on a cached side stream the
 * records instead of gathering them (the same FP32 records, summed in another order: the
 * results agree to FP32 rounding); a vertex that stays fixed over many bubbles (the full
 * vertex of a multiloop step, Sec. III.C) is then gathered once.  The cache reflects the slot's arrays when the build runs (asynchronous on
 * `stream`): rebuild it after changing their contents.  Any kb_set_vertex* call on the
 * slot, kb_set_grids, kb_set_model or kb_set_self_energy makes it stale (then unused);
 * kb_vertex_uncache frees it.
 * KB_ERR_OOM if the cache does not fit. */
kb_status kb_vertex_cache(kb_ctx *ctx, int slot, int channel, unsigned sides, void *stream);
kb_status kb_vertex_uncache(kb_ctx *ctx, int slot);

/* The full vertex of slot `slot` — its bare part and the classes of its included channels
 * (excluded channels still enter the up-up component as crossing partners), each read at
 * the point converted to its own channel variables (Sec. II.C.1) and interpolated linearly
 * in x (Sec. II.G.7) — at n points (w, v, v') in the variables of channel `channel`:
 * freqs is a DEVICE array [n][3] of doubles (±inf allowed: a class at an infinite argument
 * reads 0), out a DEVICE complex128 array [n][16] in the Keldysh order above; spin_uu != 0
 * gives the up-up component, else up-down.  E.g. the slice of the paper's post-processing:
 * channel t, w = 0, (v, v') on a grid.  Asynchronous on `stream`. */
kb_status kb_vertex_eval(kb_ctx *ctx, int slot, int channel, int spin_uu, int n, const double *freqs, void *out,
                         void *stream);

/* Self-energy loop (the paper's `loop` function, Sec. II.D.2): the vertex of slot `slot`
 * closed by one propagator line P of the context's model — which = 0: P = G; which = 1:
 * P = S, the single-scale propagator of the flow scheme (kb_set_regulator, with the
 * Katanin substitution when set), the one-loop term of the self-energy flow; which = 2:
 * P = G dSigma G, one insertion of the kb_set_self_energy_derivative tables (zero without
 * them), the line of the multiloop self-energy flow's t term; or-ed with KB_LOOP_UD_ONLY:
 * the up-down vertex alone (Gamma_s = Gamma_up-down, the Schwinger-Dyson equation's bubble
 * forms) —
 *   Sigma^{a1'|a1}(v) = - int dv'/(2 pi i) sum_{a2', a2} Gamma_s^{a1' a2'|a1 a2}(v, v'|v, v')
 *                          P^{a2|a2'}(v'),   Gamma_s = Gamma_up-down + Gamma_up-up,
 * with the vertex read in t-channel variables (w_t = 0, v, v') and the internal line's
 * spin summed (SU(2)).  The minus sign is that of the Schwinger-Dyson equation's bare term
 * (Sec. III.B): with the bare vertex -U/2 the loop of R alone is the Hartree shift
 * U (n - 1/2).  The v' integral is the symmetric principal value at v' = ±inf, on the
 * context's composite GL5 rule in x (the same nodes as the bubble) with the limits of the
 * integrand at x = ±1.  nus: DEVICE array of n doubles; out: DEVICE complex128 array
 * [n][2][2] indexed [a1'][a1] (0 classical, 1 quantum): (1,0) = Sigma^R, (0,1) = Sigma^A,
 * (1,1) = Sigma^K, (0,0) = 0 for a causal result.  Plain FP64.  Requires the grids, the
 * model and the slot.  Asynchronous on `stream`. */
enum { KB_LOOP_UD_ONLY = 4 };   /* or-ed into `which`: the up-down vertex alone (Gamma_s = Gamma_up-down) */
kb_status kb_loop(kb_ctx *ctx, int slot, int which, int n, const double *nus, void *out, void *stream);

/* Autotuning of the tensor-core K3 contraction (default off): with `on`, the first
 * mixed-precision bubble of each contraction shape (rows, columns, K, batch of bosonic
 * frequencies) times up to four split-K factors ranked by the wave model and keeps the
 * fastest for that shape and device (process-wide table); kb_graph_create tunes the shapes
 * of its bubbles before capturing.  Tuning runs extra launches on the workspace only; any
 * split-K factor gives the same result up to the rounding of the segment sums. */
kb_status kb_set_autotune(kb_ctx *ctx, int on);

/* Device workspace limit of a context in bytes (default 4 GiB, or the KB_WORKSPACE_MB
 * environment variable at kb_create).  Larger limits let the K3 contraction batch more
 * bosonic frequencies per launch; smaller ones bound memory when many contexts coexist.
 * Takes effect at the next call that sizes the workspace.  The workspace grows on demand,
 * stream-ordered on the calling stream (no device-wide synchronisation): a context's calls
 * must therefore be ordered, one stream or streams the caller orders; inside a stream
 * capture it cannot grow (KB_ERR_STATE), so size it first (kb_graph_create does). */
kb_status kb_set_workspace_limit(kb_ctx *ctx, unsigned long long bytes);

/* Synchronise the context's device and report device-side failures since the last check:
 * KB_ERR_TIMEOUT if a bounded wait inside a tensor-core kernel gave up (that kernel's output
 * is then incomplete), KB_ERR_CUDA for a CUDA error, and, in a bounds-checked build,
 * KB_ERR_STATE if a vertex record index from a frequency lookup fell outside its class (the
 * access was skipped; the message names the first one).  Clears what it reports. */
kb_status kb_check_device(kb_ctx *ctx);

/* Physical-only Keldysh structure of a vertex (Sec. II.E.2 FDRs, Sec. II.G.3 symmetries).
 * In the parquet approximation each class of channel r keeps the bare vertex's dependence on
 * the parity of the quantum indices: with a component c = (a1', a2', a1, a2) written as
 * (left pair, right pair) of the channel — a: (a1', a2), (a1, a2'); p: (a1', a2'), (a1, a2);
 * t: (a1', a1), (a2', a2) — K1 depends on the two pairs' parities only (4 distinct numbers of
 * 16), K2 on the left pair and the right parity (8), K2' on the left parity and the right
 * pair (8), K3 on both pairs (16).
 * kb_keldysh_check: residuals of these relations for the classes of `channel` in `slot`
 *   (host out[8]): out[0..3] max |X_c − X_rep(c)| / max |X| for K1, K2, K2', K3 (0 for a
 *   physical vertex; K3 is always 0; 0 for an absent class); for K1 in thermal equilibrium
 *   at temperature T, relative to max |K1|: out[4] causality (the all-even block),
 *   out[5] conjugation |K1^A − (K1^R)*| and out[6] the bosonic FDR
 *   |tanh(w/2T) K1^K − (K1^R − K1^A)| (retarded block: the one of component 1 for a and t,
 *   8 for p; advanced: its mirror; Keldysh: odd-odd); out[7] = 0.  Synchronises `stream`.
 * kb_vertex_pack: writes the distinct components of class cls (records × 4, 8, 8 or 16, the
 *   class's element type; device pointer dst, caller-owned) in the compact order d(c) = K1:
 *   2 pl + pr; K2: 4 x + 2 y + pr (x, y the left pair's indices); K2': 4 pl + 2 x' + y';
 *   K3: c — each from the smallest component c with that index.
 * kb_vertex_unpack: the class from its distinct components (the inverse for a physical
 *   vertex); overwrites the slot's class array.  Both are asynchronous on `stream`. */
kb_status kb_keldysh_check(kb_ctx *ctx, int slot, int channel, double T, double *out, void *stream);
kb_status kb_vertex_pack(kb_ctx *ctx, int slot, int channel, int cls, void *dst, void *stream);
kb_status kb_vertex_unpack(kb_ctx *ctx, int slot, int channel, int cls, const void *src, void *stream);

/* 1 if the library was compiled as the bounds-checked variant (-DKB_CHECKED: every vertex
 * record index that comes from a frequency lookup — gathers, loop, adjoint scatters — is
 * checked against its class's record count before the access; the stand-in for a memory
 * checker), else 0. */
int kb_build_checked(void);

/* Test hooks of the failure paths (no effect on results otherwise):
 * kb_inject_alloc_failures: the next n workspace allocations of this context report
 *   KB_ERR_OOM as a failed cudaMalloc would, before anything of that call is launched;
 * kb_set_wait_budget: the clock-cycle budget of the bounded wait of kb_check_wait (0
 *   restores the default, ~2 s); the tensor-core kernels keep their fixed budget of ~2 s;
 * kb_check_wait: launches one CTA that waits, with that budget, on a shared-memory barrier
 *   nothing arrives on — the wait gives up, the kernel records it in the device status and
 *   returns; the next kb_check_device reports KB_ERR_TIMEOUT and clears it, and the context
 *   stays usable.  It exercises the timeout path without any copy or MMA in flight. */
kb_status kb_inject_alloc_failures(kb_ctx *ctx, int n);
kb_status kb_set_wait_budget(kb_ctx *ctx, long long cycles);
kb_status kb_check_wait(kb_ctx *ctx, void *stream);

/* Bytes of device workspace the library currently holds (grows on demand). */
kb_status kb_workspace_bytes(kb_ctx *ctx, unsigned long long *bytes);

/* Number of kernel launches issued by this context since creation (for accounting). */
kb_status kb_launch_count(kb_ctx *ctx, unsigned long long *count);

/* Kernel timing: when enabled, every kernel launch of this context is bracketed by CUDA
 * events on its stream.  kb_profile_read aggregates the records per kernel name (after
 * synchronising the device): index i in [0, n) where n is returned in *count when name is
 * NULL; otherwise *name (static string), *ms (total device time) and *launches of entry i.
 * Enabling clears earlier records. */
kb_status kb_profile_enable(kb_ctx *ctx, int on);
kb_status kb_profile_read(kb_ctx *ctx, int index, const char **name, double *ms, unsigned long long *launches,
                          int *count);

/* ---------------------------------------------------------------------------------------
 * Allocation-free entry point.
 *
 * For callers that cannot call cudaMalloc — code running where the device memory is owned
 * by someone else (a fixed memory pool, a host program that pre-reserves all memory), or
 * code that must not trigger an allocation (and the implicit synchronisation it can cause)
 * in the middle of its own work.  This function evaluates ONE output class of the plain
 * FP64 bubble (the same kernels as kb_bubble with KB_PREC_FP64) and allocates nothing: its
 * intermediate buffers (quadrature table, Pi table, vertex tiles, contraction result) live
 * in a fixed device array of KB_NOALLOC_SCRATCH_BYTES that is part of the library image,
 * so every GPU that loads libkb holds that array until the process exits.  The paper has no
 * counterpart of this call; it is a deployment convenience.
 *
 * No context is used.  The caller passes the grids, the model (Sigma = 0: G^R = 1/(v - eps
 * + i Delta)), the two vertices as device pointers in the layout above, and the device
 * output array of class `cls` of channel `channel` (out <- alpha B + beta out).  With
 * pi_kind = KB_PI_GS_SG the single-scale propagator S is always that of the hybridisation
 * flow (S^R = -i (G^R)^2, the KB_REG_DELTA scheme of kb_set_regulator); the other flow
 * schemes need a context.  `stream` must belong to the current device (KB_ERR_ARG
 * otherwise), and the call refuses to start (KB_ERR_CUDA) while an earlier launch error is
 * pending on this thread; it returns at the first chunk whose launches fail.
 * The first call on a device looks up the array's device address (and uploads the small
 * index tables); make that first call before any stream capture.  All calls share the one
 * array, and each call overwrites every scratch element it reads, so no call depends on an
 * earlier one; calls whose work overlaps on the GPU (different streams, or different host
 * threads, without ordering between them) race on the array and must be serialised by the
 * caller.  The work runs in bosonic-frequency chunks that fit the array; a problem whose
 * single bosonic frequency does not fit (roughly (8 n_v nq (2 for t)) * 16 bytes for the
 * vertex tiles) returns KB_ERR_TOO_LARGE without launching anything.
 * --------------------------------------------------------------------------------------- */
#define KB_NOALLOC_SCRATCH_BYTES (32u << 20)

typedef struct {
    int has_R;              /* include the bare vertex R = Gamma0 */
    double U;               /* its strength */
    unsigned channels;      /* included channels (bits), as kb_set_vertex_channels */
    const void *cls[3][4];  /* device pointers [channel][K1, K2, K2', K3], NULL = absent */
    int dtype[3][4];        /* KB_DT_C128 / KB_DT_C64 */
} kb_vertex_desc;

kb_status kb_bubble_fp64_noalloc(const kb_grid_desc *g, double Delta, double T, double eps,
                                 const kb_vertex_desc *left, const kb_vertex_desc *right, int channel,
                                 int pi_kind, int cls, void *out, int out_dtype, double alpha, double beta,
                                 void *stream);

/* Susceptibilities from the K1 class of channel `channel` of a slot (the paper's
 * post-processing, Sec. II.E.5: K1_r = R χ_r R for a converged parquet vertex, R = -U/2 on
 * the components with an odd number of quantum indices), on the K1 grid, into the DEVICE
 * array `out` of n1 x 2 complex doubles [w][χ^R, χ^K]:
 *   KB_CH_A  transverse spin, χ = -2 K1_a / U² on the retarded (component 1) and Keldysh (3)
 *            blocks;
 *   KB_CH_P  pairing, χ = +2 K1_p / U² (components 8 and 9);
 *   KB_CH_T  charge, both spins of the pair: χ = 2 [K1_t(ω) + K1_t^uu(ω)] / U² with
 *            K1_t^uu(ω) = K1_t(ω) - K1_a(-ω), a1 <-> a2 swapped (needs the slot's a-channel K1).
 * At second order these are the bare bubbles (-Π_ph/2, Π_pp/2, -Π_ph/2).  With U = 1 the same
 * readout gives the leg contraction from the K1 of a bubble chain closed by a unit bare vertex
 * (R̂ Π R̂ + R̂ Π Γ Π R̂, built from kb_bubble calls).  K1 in c128 or c64; asynchronous on
 * `stream`. */
kb_status kb_susceptibility_k1(kb_ctx *ctx, int channel, int slot, double U, void *out, void *stream);

/* Human-readable description of the last error on this context (never NULL). */
const char *kb_last_error(kb_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* KB_H */
