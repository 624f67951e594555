"""Pins of the FP64 oracle against facts fixed outside itself.

Closed forms (RMSNorm, SiLU, SwiGLU, attention special cases, Gaussian
likelihood), the paper's Fig. 2 grids transcribed by hand, window-mask
cardinalities, schedule step counts, a dense-mask NumPy formulation of the
model on tiny frames, schedule equivalence, brute-force causality, CDF table
invariants, rANS round trips and size bounds, E4M3 rounding (hand values of
the format, a library cast), and the data generator's statistics.  CPU only.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import dense_ref
from paper_2605_20977_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    for line in open(os.path.join(GOLDEN, name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append(line.split())
    return rows


# ----------------------------------------------------------- elementary ops

def test_rmsnorm_closed_form():
    # x = (3, 4): mean square 12.5
    y = O.rmsnorm([3.0, 4.0], [1.0, 2.0])
    s = math.sqrt(12.5 + 1e-6)
    assert y == pytest.approx([3.0 / s, 8.0 / s], rel=1e-15)
    # a constant vector maps to the gain (up to eps)
    y = O.rmsnorm([5.0] * 8, np.arange(8.0))
    assert y == pytest.approx(np.arange(8.0) * 5.0 / math.sqrt(25.0 + 1e-6), rel=1e-15)


def test_silu_closed_forms():
    assert O.silu(0.0) == 0.0
    assert O.silu(1.0) == pytest.approx(1.0 / (1.0 + math.exp(-1.0)), rel=1e-15)
    for x in (-3.0, -0.5, 0.25, 2.0, 7.0):          # x s(x) - (-x) s(-x) = x
        assert O.silu(x) - O.silu(-x) == pytest.approx(x, rel=1e-14)


def test_matvec_matches_library_matmul():
    rng = np.random.default_rng(0)
    x = rng.standard_normal(17); W = rng.standard_normal((17, 5))
    assert O.matvec(x, W) == pytest.approx(x @ W, rel=1e-13, abs=1e-13)
    # orientation: x . W with W [in][out]; a unit x picks a row of W
    e = np.zeros(17); e[3] = 1.0
    assert np.array_equal(O.matvec(e, W), W[3])


def test_swiglu_closed_form():
    # d = F = 1: out = silu(x g) (x u) dw
    out = O.swiglu([2.0], [[0.5]], [[3.0]], [[-1.5]])
    assert out[0] == pytest.approx(O.silu(1.0) * 6.0 * -1.5, rel=1e-15)
    # zero gate projection gives zero output
    rng = np.random.default_rng(1)
    x = rng.standard_normal(6)
    assert np.all(O.swiglu(x, np.zeros((6, 4)), rng.standard_normal((6, 4)), rng.standard_normal((4, 6))) == 0.0)


def test_attention_special_cases():
    rng = np.random.default_rng(2)
    d, nh = 8, 2
    q = rng.standard_normal(d)
    K = rng.standard_normal((3, d)); V = rng.standard_normal((3, d))
    bias = rng.standard_normal((3, nh))
    # one key: the output is that key's value row
    assert O.attend(q, K[:1], V[:1], bias[:1], nh) == pytest.approx(V[0], rel=1e-15)
    # zero query and zero bias: uniform average of the values
    assert O.attend(np.zeros(d), K, V, np.zeros((3, nh)), nh) == pytest.approx(V.mean(0), rel=1e-14)
    # empty key set: zero
    assert np.all(O.attend(q, K[:0], V[:0], bias[:0], nh) == 0.0)
    # two keys: per head the weight of key 0 is a logistic of the score gap
    out = O.attend(q, K[:2], V[:2], bias[:2], nh)
    dh = d // nh
    for h in range(nh):
        sl = slice(h * dh, (h + 1) * dh)
        s0 = q[sl] @ K[0, sl] / math.sqrt(dh) + bias[0, h]
        s1 = q[sl] @ K[1, sl] / math.sqrt(dh) + bias[1, h]
        p0 = 1.0 / (1.0 + math.exp(s1 - s0))
        assert out[sl] == pytest.approx(p0 * V[0, sl] + (1 - p0) * V[1, sl], rel=1e-12, abs=1e-14)
    # a dominant bias selects its key
    big = np.zeros((3, nh)); big[2] = 1e3
    assert O.attend(q, K, V, big, nh) == pytest.approx(V[2], rel=1e-12)


# ----------------------------------------------------------- masks, schedules

def test_fig2a_cyclic_labels_golden():
    g = _golden("fig2a_labels.txt")
    for a, row in enumerate(range(-2, 6)):
        for b, col in enumerate(range(-2, 6)):
            # shift by one period so indices are non-negative; the pattern repeats every 4
            assert O.label(1, row + 4, col + 4) + 1 == int(g[a][b]), (row, col)


def test_fig2b_receptive_field_golden():
    g = _golden("fig2b_receptive_field.txt")
    ti, tj = 1 + 4, 1 + 4          # target (1, 1) shifted by one period
    W = 12
    for a, di in enumerate(range(-2, 3)):
        for b, dj in enumerate(range(-2, 3)):
            qi, qj = ti + di, tj + dj
            acc = O.visible(1, 0, W, ti, tj, qi, qj)
            sa = O.visible(1, 1, W, ti, tj, qi, qj)
            want = g[a][b]
            assert acc == (want == "A"), (di, dj)
            assert sa == (want in ("A", "S", "T")), (di, dj)


@pytest.mark.parametrize("k,nS,nA", [(5, 13, 11), (7, 24, 22)])
def test_wavefront_mask_interior_counts(k, nS, nA):
    c = synth.config("i1080") if k == 7 else synth.config("tiny").with_grid(16, 16)
    p = 10 * c.W + 10
    assert len(O.window_keys(c, 1, p)[0]) == nS
    assert len(O.window_keys(c, 0, p)[0]) == nA
    # accumulator keys have smaller label and raster index; S adds p and same-step keys
    idx, _ = O.window_keys(c, 1, p)
    pi, pj = divmod(p, c.W)
    for q in idx:
        qi, qj = divmod(int(q), c.W)
        assert 2 * qi + qj <= 2 * pi + pj and q <= p


def test_wavefront_same_step_keys_k7():
    # only (i-1, j+2) shares the step and precedes in raster order (Sec. 3.2:
    # same-step positions are visible to self-attention, not to the accumulator)
    c = synth.config("i1080")
    p = 30 * c.W + 40
    s_only = set(O.window_keys(c, 1, p)[0].tolist()) - set(O.window_keys(c, 0, p)[0].tolist())
    assert s_only == {p, 29 * c.W + 42}


def test_schedule_step_counts():
    c = synth.config("tiny")
    order, start = O.schedule(c, 0)
    assert len(start) - 1 == 2 * (c.H - 1) + (c.W - 1) + 1 == 26
    assert sorted(order.tolist()) == list(range(c.H * c.W))
    _, start = O.schedule(c, 1)
    assert len(start) - 1 == 96
    c = synth.config("i1080")
    order, start = O.schedule(c, 0)
    assert len(start) - 1 == 254
    assert max(np.diff(start)) == 60
    _, start = O.schedule(c, 1)
    assert len(start) - 1 == 8160
    # cyclic s = 4: four steps regardless of resolution (Sec. 2, Sec. 3.2)
    for nm in ("tiny_cyc", "i1080_cyc"):
        cc = synth.config(nm)
        assert len(O.schedule(cc, 0)[1]) - 1 == 4
        _, st = O.schedule(cc.with_grid(68, 120), 0)
        assert len(st) - 1 == 4 and np.diff(st).tolist() == [2040] * 4


# ----------------------------------------------------------- model

@pytest.mark.parametrize("name,vary", [(n, False) for n in ("tiny", "tiny_cyc", "tiny_p", "tiny_ct", "tiny_cyc_ct",
                                                              "tiny_p_ct")] +
                         [("tiny", True), ("tiny_p", True), ("tiny_cyc_ct", True)])
def test_oracle_matches_dense_mask_formulation(name, vary):
    """The whole model against full [HW x HW] attention under the masks.
    With vary, every channel-wise scale and offset (input and context
    embedding scales, the Channel Transformer's latent scales, the heads'
    output scales and offsets) differs per channel, so a wrong channel index
    or a dropped offset shows."""
    c = synth.config(name)
    w = synth.weights(c, vary_consts=vary)
    fr = synth.frames(c, 3 if c.temporal else 1, seed=7)
    mu0, s0 = O.run(c, w, fr.y, fr.z, driver=0)
    mu1, s1 = dense_ref.run(c, w, fr.y, fr.z)
    assert np.max(np.abs(mu0 - mu1)) < 1e-11
    assert np.max(np.abs(np.log(s0) - np.log(s1))) < 1e-11


@pytest.mark.parametrize("name", ["tiny", "tiny_cyc", "tiny_ct", "tiny_hp"])
def test_translation_equivariance_downwards(name):
    """The same for a shift of 4 rows down (hyperlatents 4 / r rows): every
    row whose dependencies stay clear of the top and bottom borders in both
    frames (the model's reach, 10 rows, each way: the cyclic mask sees lower
    labels below a position, and the convolutional hyperprior's synthesis
    reaches below it) shifts with the latents, bit for bit, across the whole
    width."""
    c = synth.config(name).with_grid(32, 16)
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=52)
    s, sz = 4, 4 // c.r
    y2 = np.zeros_like(fr.y)
    y2[:, s:] = fr.y[:, :-s]
    z2 = np.zeros_like(fr.z)
    z2[:, sz:] = fr.z[:, :-sz]
    mu0, s0 = O.run(c, w, fr.y, fr.z, driver=0)
    mu1, s1 = O.run(c, w, y2, z2, driver=0)
    rows = np.arange(10, c.H - s - 10)
    assert np.array_equal(mu1[0][rows + s], mu0[0][rows]) and np.array_equal(s1[0][rows + s], s0[0][rows])
    assert not np.array_equal(mu0[0][rows + s], mu0[0][rows])


@pytest.mark.parametrize("name", ["tiny", "tiny_cyc", "tiny_ct", "tiny_hp"])
def test_translation_equivariance_away_from_borders(name):
    """Window attention with relative biases under masks that depend only on
    relative offsets (2i+j: label differences and, within a label, the
    raster order; cyclic: labels of period 4): shifting the latents right by
    4 columns and the hyperlatents by 4 / r shifts every parameter by 4
    columns, bit for bit, wherever neither frame's border lies within the
    model's reach (L w + w + L w = 10 columns here; 12 kept clear)."""
    c = synth.config(name).with_grid(8, 44)
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=51)
    s, sz = 4, 4 // c.r
    y2 = np.zeros_like(fr.y)
    y2[:, :, s:] = fr.y[:, :, :-s]
    z2 = np.zeros_like(fr.z)
    z2[:, :, sz:] = fr.z[:, :, :-sz]
    mu0, s0 = O.run(c, w, fr.y, fr.z, driver=0)
    mu1, s1 = O.run(c, w, y2, z2, driver=0)
    cols = np.arange(12, c.W - s - 12)
    assert np.array_equal(mu1[0][:, cols + s], mu0[0][:, cols])
    assert np.array_equal(s1[0][:, cols + s], s0[0][:, cols])
    # the comparison is not vacuous: the parameters differ between columns
    assert not np.array_equal(mu0[0][:, cols + s], mu0[0][:, cols])


@pytest.mark.parametrize("name", ["tiny", "tiny_ct"])
def test_heads_sigma_clamped_at_both_ends(name):
    """sigma = exp of the scaled head output clamped to [ln 0.11, ln 256]
    (Sec. 3.1 heads; the scale table's range): with the offsets of some
    channels far below and of others far above the range, those channels
    come out at exactly the clamp values and the rest as the dense
    formulation gives them (the plain heads and the grouped heads)."""
    c = synth.config(name)
    w = synth.weights(c).astype(np.float64)
    off = 0
    for t in synth.weight_spec(c):
        if t.name == "beta_sig":
            break
        off += int(np.prod(t.shape))
    lo_ch, hi_ch = np.arange(0, c.C, 4), np.arange(1, c.C, 4)
    w[off + lo_ch] = -12.0
    w[off + hi_ch] = 14.0
    fr = synth.frames(c, 1, seed=9)
    mu0, s0 = O.run(c, w, fr.y, fr.z, driver=0)
    mu1, s1 = dense_ref.run(c, w, fr.y, fr.z)
    assert np.all(s0[..., lo_ch] == math.exp(math.log(0.11)))
    assert np.all(s0[..., hi_ch] == math.exp(math.log(256.0)))
    assert np.max(np.abs(mu0 - mu1)) < 1e-11
    assert np.max(np.abs(np.log(s0) - np.log(s1))) < 1e-11


@pytest.mark.parametrize("grid", [None, (5, 7), (1, 9)])
def test_lrp_oracle_matches_dense_mask_formulation(grid):
    """The LRP Transformer's residual (Sec. 3.1): the oracle's per-position
    window loops against full [HW x HW] attention under the unmasked window
    mask, on the model's own representation; a full and two ragged grids."""
    c = synth.config("tiny_lrp")
    if grid:
        c = c.with_grid(*grid)
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=13)
    mu0, s0, e0 = O.run(c, w, fr.y, fr.z, driver=0, with_eps=True)
    mu1, s1, e1 = dense_ref.run(c, w, fr.y, fr.z, with_eps=True)
    assert np.max(np.abs(mu0 - mu1)) < 1e-11
    assert np.max(np.abs(e0 - e1)) < 1e-11
    # the LRP leaves the entropy model's parameters as they are
    c0 = synth.config("tiny")
    if grid:
        c0 = c0.with_grid(*grid)
    mu2, s2 = O.run(c0, w[:synth.weights_count(c0)], fr.y, fr.z, driver=0)
    assert np.array_equal(mu0, mu2) and np.array_equal(s0, s2)


def test_lrp_temporal_oracle_matches_dense_mask_formulation():
    """The temporal model's LRP Transformer (time-causal: windows of the
    current and Tf - 1 previous frames, bias by frame age) over four frames,
    so that the three-frame ring wraps: the oracle's ring of per-block keys
    and values against dense attention over the concatenated frames."""
    c = synth.config("tiny_p_lrp")
    w = synth.weights(c, vary_consts=True)       # the LRP's latent scales per channel
    fr = synth.frames(c, 4, seed=16)
    mu0, s0, e0 = O.run(c, w, fr.y, fr.z, driver=0, with_eps=True)
    mu1, s1, e1 = dense_ref.run(c, w, fr.y, fr.z, with_eps=True)
    assert np.max(np.abs(mu0 - mu1)) < 1e-11
    assert np.max(np.abs(e0 - e1)) < 1e-11
    # a latent of frame 0 reaches the residual of frames 1 and 2 (through
    # the LRP ring as well as the temporal entropy model) but a latent of
    # frame 2 leaves frames 0 and 1 as they are (time-causal)
    y = fr.y.copy()
    y[2, 3, 4, :] += 5
    _, _, e2 = O.run(c, w, y, fr.z, driver=0, with_eps=True)
    assert np.array_equal(e2[:2], e0[:2]) and not np.array_equal(e2[2], e0[2])


def test_lrp_residual_is_the_same_after_decoding():
    """Decoding the frame from its container (the wavefront schedule
    revealing latents step by step) gives bit-for-bit the residual of the
    masked pass: the LRP runs on the coded latents and final
    representations only."""
    c = synth.config("tiny_lrp")
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=14)
    _, _, e0 = O.run(c, w, fr.y, fr.z, driver=0, with_eps=True)
    bs, _, _ = O.encode_frames(c, w, fr.y, fr.z)
    y = np.zeros_like(fr.y)
    _, _, e2 = O.run(c, w, y, fr.z, driver=2, bitstreams=bs, with_eps=True)
    assert np.array_equal(y, fr.y)
    assert np.array_equal(e0, e2)


def test_lrp_window_is_spatially_unmasked_and_local():
    """Perturbing the latent at q: the entropy parameters move at a set S of
    positions after q in raster order (within 2L+1 window radii: L Spatial
    Module 1 blocks, the accumulator, L Spatial Module 2 blocks), and the
    LRP residual moves exactly on the Llrp-radius Chebyshev dilation of
    S and q (unmasked k x k windows, Llrp blocks, clipped at the border):
    in every direction, positions before q included."""
    c = synth.config("tiny_lrp").with_grid(20, 40)
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=15)
    mu0, _, e0 = O.run(c, w, fr.y, fr.z, driver=0, with_eps=True)
    qi, qj = 10, 20
    y = fr.y.copy()
    y[0, qi, qj, :] += 7
    mu1, _, e1 = O.run(c, w, y, fr.z, driver=0, with_eps=True)
    moved = np.abs(e1 - e0).max(axis=-1)[0] > 0
    S = np.abs(mu1 - mu0).max(axis=-1)[0] > 0
    R = (c.k - 1) // 2
    ii, jj = np.meshgrid(np.arange(c.H), np.arange(c.W), indexing="ij")
    rho, rq = ii * c.W + jj, qi * c.W + qj
    G = (2 * c.L + 1) * R
    assert S.any() and not S[(rho <= rq) | (np.abs(ii - qi) > G) | (np.abs(jj - qj) > G)].any()
    reach = np.zeros_like(S)
    for a, b in zip(*np.nonzero(S | (rho == rq))):
        reach |= (np.abs(ii - a) <= c.Llrp * R) & (np.abs(jj - b) <= c.Llrp * R)
    assert (~reach).any() and np.array_equal(moved, reach)
    assert moved[(rho < rq)].any()


def test_weight_layout_count_matches_generator():
    for nm in ("tiny", "tiny_p", "i1080", "p1080", "tiny_lrp", "i1080_lrp", "tiny_p_lrp", "p1080_lrp",
               "tiny_ct", "tiny_p_ct", "tiny_ct_lrp", "i1080_ct", "i1080_cyc_ct", "tiny_hp", "i1080_hp", "p1080_hp"):
        c = synth.config(nm)
        assert O.weights_count(c) == synth.weights_count(c)


@pytest.mark.parametrize("name,sched", [("tiny", 0), ("tiny", 1), ("tiny_cyc", 0), ("tiny_p", 0), ("tiny_p", 1),
                                        ("tiny_ct", 0), ("tiny_ct", 1), ("tiny_cyc_ct", 0), ("tiny_p_ct", 0)])
def test_schedules_give_the_masked_pass_bit_exact(name, sched):
    c = synth.config(name)
    w = synth.weights(c)
    fr = synth.frames(c, 3 if c.temporal else 1, seed=11)
    mu0, s0 = O.run(c, w, fr.y, fr.z, driver=0)
    mu1, s1 = O.run(c, w, fr.y, fr.z, driver=1, sched=sched)
    assert np.array_equal(mu0, mu1) and np.array_equal(s0, s1)


def _closure(c):
    """dep[p] = positions whose latent can reach params(p): S^L(A(S^L(p)))."""
    _, A, S, _ = dense_ref.grid_masks(c)
    HW = c.H * c.W
    Si = S.astype(np.int64)
    reach = np.eye(HW, dtype=np.int64)
    for _ in range(c.L):
        reach = (reach @ Si > 0).astype(np.int64)
    reach = (reach @ A.astype(np.int64) > 0).astype(np.int64)
    for _ in range(c.L):
        reach = (reach @ Si > 0).astype(np.int64)
    return reach > 0


def test_causality_brute_force():
    # perturb the latent at each q and record which parameters change
    c = synth.config("tiny")
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=3)
    mu0, s0 = O.run(c, w, fr.y, fr.z)
    dep = _closure(c)
    HW = c.H * c.W
    lab = np.array([2 * (p // c.W) + p % c.W for p in range(HW)])
    for q in range(HW):
        y = fr.y.copy()
        y[0].reshape(HW, c.C)[q] += 5
        mu, s = O.run(c, w, y, fr.z)
        changed = np.any((mu != mu0) | (s != s0), axis=-1).reshape(HW)
        assert np.array_equal(changed, dep[:, q]), q
        assert np.all(lab[changed] > lab[q]) and np.all(np.nonzero(changed)[0] > q)


def test_channel_groups_causal_within_a_position():
    """Channel Transformer (Sec. 3.1): perturbing the latents of channel
    group g at position q leaves the parameters of groups 0..g at q as they
    were and moves those of group g + 1 (the channel shift feeds group g's
    latents to group g + 1 only; the block-lower-triangular mixing passes
    them on to later groups); group 0 at q depends on no latent of q."""
    c = synth.config("tiny_ct")
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=19)
    mu0, s0 = O.run(c, w, fr.y, fr.z)
    Cg = c.C // c.Nc
    qi, qj = 3, 5
    for g in range(c.Nc):
        y = fr.y.copy()
        y[0, qi, qj, g * Cg:(g + 1) * Cg] += 6
        mu, s = O.run(c, w, y, fr.z)
        moved = np.any((mu[0, qi, qj] != mu0[0, qi, qj]).reshape(c.Nc, Cg) |
                       (s[0, qi, qj] != s0[0, qi, qj]).reshape(c.Nc, Cg), axis=1)
        assert not moved[:g + 1].any(), g
        if g + 1 < c.Nc:
            assert moved[g + 1:].all(), g
    y = fr.y.copy()
    y[0, qi, qj, :] -= 4
    mu, s = O.run(c, w, y, fr.z)
    assert np.array_equal(mu[0, qi, qj, :Cg], mu0[0, qi, qj, :Cg])
    assert np.array_equal(s[0, qi, qj, :Cg], s0[0, qi, qj, :Cg])


def test_channel_transformer_lrp_on_its_output():
    """The LRP Transformer of a model with a Channel Transformer reads the
    Channel Transformer's stream (the heads' input): oracle against the
    dense formulation."""
    c = synth.config("tiny_ct_lrp")
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=20)
    _, _, e0 = O.run(c, w, fr.y, fr.z, driver=0, with_eps=True)
    _, _, e1 = dense_ref.run(c, w, fr.y, fr.z, with_eps=True)
    assert np.max(np.abs(e0 - e1)) < 1e-11
    _, _, e2 = O.run(c, w, fr.y, fr.z, driver=1, with_eps=True)
    assert np.array_equal(e0, e2)


# ----------------------------------------------------------- hyperprior

@pytest.mark.parametrize("name,grid,vary", [("tiny_hp", None, False), ("tiny_p_hp", None, True),
                                           ("i1080_hp", (9, 14), False)])
def test_hyperprior_matches_dense_formulation(name, grid, vary):
    """Convolutional hyperprior (Fig. 1 right): the oracle's analysis (z
    from the Spatial Module 1 output through the RB-down blocks) and its
    synthesis (the hyperprior tokens from z-hat through the RB-up blocks,
    cropped) against a NumPy formulation by shifted views and a reshape
    pixel shuffle; 9 x 14 is ragged (hyperprior grid 3 x 4, synthesis grid
    12 x 16 cropped).  z-hat is z rounded half to even."""
    c = synth.config(name)
    if grid:
        c = c.with_grid(*grid)
    w = synth.weights(c, vary_consts=vary)      # vary: the z-hat scales per channel as well
    fr = synth.frames(c, 2 if c.temporal else 1, seed=21)
    zh, z = O.hyper_analysis(c, w, fr.y)
    assert np.array_equal(zh, np.rint(z).astype(np.int16))
    mu0, s0 = O.run(c, w, fr.y, zh, driver=0)
    mu1, s1, z1 = dense_ref.run(c, w, fr.y, zh, with_z=True)
    assert np.max(np.abs(z - z1)) < 1e-11
    assert np.max(np.abs(mu0 - mu1)) < 1e-11 and np.max(np.abs(np.log(s0) - np.log(s1))) < 1e-11


def test_hyperprior_model_schedules_and_round_trip():
    """With the convolutional hyperprior the wavefront decode reproduces the
    masked pass bit for bit and the container round trip is lossless."""
    c = synth.config("tiny_hp")
    w = synth.weights(c)
    fr = synth.frames(c, 1, seed=22)
    zh, _ = O.hyper_analysis(c, w, fr.y)
    mu0, s0 = O.run(c, w, fr.y, zh, driver=0)
    mu1, s1 = O.run(c, w, fr.y, zh, driver=1)
    assert np.array_equal(mu0, mu1) and np.array_equal(s0, s1)
    bs, mu, sg = O.encode_frames(c, w, fr.y, zh)
    yd, mud, sgd = O.decode_frames(c, w, bs, zh)
    assert np.array_equal(yd, fr.y) and np.array_equal(mu, mud)


def _softplus(x):
    return np.log1p(np.exp(x))


def test_factorized_prior_closed_form_without_gating():
    """With every gate a_k = 0 the cumulative is the logistic
    sigmoid(alpha x + beta) of the composed affine maps (alpha the product of
    the softplus matrices, beta the propagated biases): the oracle's rate of
    a z-hat equals the closed form; and the tables sum to 2^16 with every
    slot at least 1, close to the prior's probabilities."""
    c = synth.config("tiny_hp")
    w = synth.weights(c).astype(np.float64)
    P = dense_ref.split_weights(c, w)
    off, offs = 0, {}
    for t in synth.weight_spec(c):
        offs[t.name] = off
        off += int(np.prod(t.shape))
    for k in (1, 2, 3):
        n = int(np.prod(P[f"hp.fp_a{k}"].shape))
        w[offs[f"hp.fp_a{k}"]:offs[f"hp.fp_a{k}"] + n] = 0.0
    P = dense_ref.split_weights(c, w)
    rng = np.random.default_rng(5)
    zh = rng.integers(-6, 7, size=(c.Hh, c.Wh, c.Ch)).astype(np.int16)
    bits = 0.0
    for ch in range(c.Ch):
        H1 = _softplus(P["hp.fp_H1"][ch]).reshape(3, 1); b1 = P["hp.fp_b1"][ch]
        H2 = _softplus(P["hp.fp_H2"][ch]); b2 = P["hp.fp_b2"][ch]
        H3 = _softplus(P["hp.fp_H3"][ch]); b3 = P["hp.fp_b3"][ch]
        H4 = _softplus(P["hp.fp_H4"][ch]).reshape(1, 3); b4 = P["hp.fp_b4"][ch]
        alpha = float((H4 @ H3 @ H2 @ H1)[0, 0])
        beta = float((H4 @ (H3 @ (H2 @ b1 + b2) + b3))[0] + b4)
        sig = lambda x: 1.0 / (1.0 + np.exp(-(alpha * x + beta)))
        v = zh[..., ch].astype(np.float64)
        p = np.maximum(sig(v + 0.5) - sig(v - 0.5), 1e-9)
        bits -= np.log2(p).sum()
        f = O.prior_freq(c, w, ch)
        assert f.sum() == 1 << 16 and f.min() >= 1 and len(f) == 64
        T = 31
        pm = np.array([sig(k + 0.5) - sig(k - 0.5) for k in range(-T, T + 1)])
        assert np.max(np.abs(f[:-1] / 65536.0 - pm)) < 2e-3
    assert abs(O.hyper_rate(c, w, zh) - bits) <= 1e-9 * bits


def test_factorized_prior_table_rule_on_a_wide_prior():
    """The z-hat tables' rule, slot by slot, on a prior wide and off-centre
    enough that both tails beyond +-31.5 carry many counts: with the gates
    at 0 and every softplus matrix entry at 0.25 the cumulative is
    sigmoid(alpha x + beta) (alpha ~ 0.1), and slot v gets
    1 + floor(P(v) (2^16 - 64)), the escape slot the same of both tails,
    slot 0 the remainder (within one where P (2^16 - 64) lies within 1e-6
    of an integer)."""
    c = synth.config("tiny_hp")
    w = synth.weights(c).astype(np.float64)
    P = dense_ref.split_weights(c, w)
    off, offs = 0, {}
    for t in synth.weight_spec(c):
        offs[t.name] = off
        off += int(np.prod(t.shape))

    def put(name, value):
        n = int(np.prod(P[name].shape))
        w[offs[name]:offs[name] + n] = value

    raw = math.log(math.expm1(0.25))                 # softplus(raw) = 0.25
    for k in (1, 2, 3):
        put(f"hp.fp_a{k}", 0.0)
    for k in (1, 2, 3, 4):
        put(f"hp.fp_H{k}", raw)
        put(f"hp.fp_b{k}", 0.0)
    put("hp.fp_b4", 1.5)
    alpha, beta = 27 * 0.25 ** 4, 1.5
    sig = lambda x: 1.0 / (1.0 + np.exp(-(alpha * x + beta)))
    T, n = 31, 64
    v = np.arange(-T, T + 1, dtype=np.float64)
    p = np.append(sig(v + 0.5) - sig(v - 0.5), sig(-T - 0.5) + (1.0 - sig(T + 0.5)))
    x = p * (65536 - n)
    want = 1 + np.floor(x).astype(np.int64)
    near = np.abs(x - np.rint(x)) < 1e-6
    rest = np.ones(n, bool)
    rest[T] = False
    assert sig(-T - 0.5) * 65536 > 100 and (1.0 - sig(T + 0.5)) * 65536 > 100
    for ch in (0, c.Ch - 1):
        f = O.prior_freq(c, w, ch).astype(np.int64)
        assert np.array_equal(f[rest & ~near], want[rest & ~near])
        assert np.all(np.abs(f[rest & near] - want[rest & near]) <= 1)
        assert f[T] == 65536 - f[rest].sum()


def test_zhat_coder_round_trip_escapes_and_corruption():
    """The z-hat container: lossless for values inside and far outside the
    table support (escapes, int16 extremes), and a flipped byte or a
    truncation is reported."""
    c = synth.config("tiny_hp")
    w = synth.weights(c)
    rng = np.random.default_rng(6)
    zh = rng.integers(-4, 5, size=(c.Hh, c.Wh, c.Ch)).astype(np.int16)
    zh[0, 0, :4] = [-32768, 32767, 40, -33]
    bs = O.hyper_encode(c, w, zh)
    ok, zd = O.hyper_decode(c, w, bs)
    assert ok and np.array_equal(zd, zh)
    bad = bytearray(bs)
    bad[len(bad) // 2] ^= 0x5A
    ok2, zd2 = O.hyper_decode(c, w, bytes(bad))
    ok3, _ = O.hyper_decode(c, w, bs[:-8])
    assert not ok2 or not np.array_equal(zd2, zh)
    assert not ok3


# ----------------------------------------------------------- rate, tables

def test_likelihood_closed_forms():
    # mu = 0, sigma = 1, y = 0: erf(1 / (2 sqrt 2))
    assert O.likelihood(0, 0.0, 1.0) == pytest.approx(0.38292492254802624, rel=1e-15)
    rng = np.random.default_rng(4)
    for _ in range(20):
        mu = rng.uniform(-5, 5); sg = math.exp(rng.uniform(math.log(0.11), math.log(60)))
        # masses of adjacent unit bins telescope to a Gaussian interval mass
        # (stay above the 1e-9 floor)
        a = b = round(mu)
        while O.likelihood(a - 1, mu, sg) > 1e-7:
            a -= 1
        while O.likelihood(b + 1, mu, sg) > 1e-7:
            b += 1
        tot = sum(O.likelihood(y, mu, sg) for y in range(a, b + 1))
        r2 = sg * math.sqrt(2.0)
        want = 0.5 * (math.erf((b + 0.5 - mu) / r2) - math.erf((a - 0.5 - mu) / r2))
        assert tot == pytest.approx(want, abs=1e-13)
        assert want > 1 - 1e-5
        u = rng.integers(0, 5)
        assert O.likelihood(round(mu) + u, round(mu), sg) == O.likelihood(round(mu) - u, round(mu), sg)
    assert O.likelihood(1000, 0.0, 1.0) == 1e-9            # floor
    assert O.likelihood(0, 0.0, 1e-3) == O.likelihood(0, 0.0, 0.11)   # clamp


def test_rate_bits_sum():
    y = np.array([0, 1, -2], np.int16)
    mu = np.array([0.0, 0.3, -1.0]); sg = np.array([1.0, 2.0, 0.5])
    want = -sum(math.log2(O.likelihood(a, b, s)) for a, b, s in zip(y, mu, sg))
    assert O.rate_bits(y, mu, sg) == pytest.approx(want, rel=1e-15)


# ----------------------------------------------------------- E4M3

def test_e4m3_hand_values():
    """Values fixed by the format (3 mantissa bits, bias 7, largest finite
    448, smallest subnormal 2^-9) and its ties-to-even rounding."""
    cases = {1.0: 1.0, 1.0625: 1.0, 1.1875: 1.25, 1.124: 1.125, -3.3: -3.25, 448.0: 448.0, 460.0: 448.0,
             1000.0: 448.0, 240.0: 240.0, 248.0: 256.0, 2.0 ** -6: 2.0 ** -6, 2.0 ** -9: 2.0 ** -9,
             2.0 ** -10: 0.0, 3 * 2.0 ** -10: 2.0 ** -8, 0.7 * 2.0 ** -9: 2.0 ** -9, 5 * 2.0 ** -10: 2.0 ** -8,
             0.0: 0.0, 17.0: 16.0, 19.0: 20.0}
    for x, want in cases.items():
        assert O.e4m3(x) == want, (x, O.e4m3(x), want)


def test_e4m3_matches_library_cast():
    """Nearest-even E4M3 of float32 values across the whole finite range,
    subnormals and exact ties included, against torch's float8_e4m3fn cast."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    mags = np.exp2(rng.uniform(-12, np.log2(440.0), 20000))
    x = (mags * rng.choice([-1.0, 1.0], mags.size)).astype(np.float32)
    grid = torch.arange(256, dtype=torch.uint8).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    grid = np.unique(grid[np.isfinite(grid) & (np.abs(grid) <= 256)])
    ties = ((grid[1:] + grid[:-1]) / 2).astype(np.float32)             # midpoints, exact in float32
    x = np.concatenate([x, ties, grid.astype(np.float32)])
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    got = np.array([O.e4m3(float(v)) for v in x])
    assert np.array_equal(got, ref)


def test_e4m3_tensor_scale_rule():
    rng = np.random.default_rng(12)
    for scale in (1e-3, 0.05, 1.0, 37.0):
        x = rng.standard_normal(4096) * scale
        q, s = O.e4m3_tensor(x)
        assert s == 2.0 ** round(math.log2(s))                        # a power of two
        assert 128.0 <= np.abs(x).max() / s < 256.0
        assert np.array_equal(q / s, [O.e4m3(v) for v in x / s])
        rel = np.abs(q - x)[np.abs(x) > 2 ** -6 * s] / np.abs(x)[np.abs(x) > 2 ** -6 * s]
        assert rel.max() <= 2.0 ** -4                                 # half a unit of 3 mantissa bits
    q, s = O.e4m3_tensor(np.zeros(8))
    assert s == 1.0 and not q.any()


def test_scale_table():
    t = O.scale_table()
    assert t[0] == np.float32(0.11) and t[-1] == np.float32(256.0)
    r = np.log(t.astype(np.float64))
    assert np.allclose(np.diff(r), (math.log(256) - math.log(0.11)) / 63, rtol=1e-6)


def test_quantize_rules():
    t = O.scale_table()
    sig = np.array([t[5], np.nextafter(t[5], np.float32(1e9)), 0.01, 1e6, t[0], np.float32("nan")], np.float32)
    idx, _ = O.quantize(np.zeros(6, np.float32), sig)
    assert idx.tolist() == [5, 6, 0, 63, 0, 63]
    mu = np.array([0.5, 1.5, -0.5, 2.5, -2.5, 1e9, -1e9, 0.49999997], np.float32)
    _, m = O.quantize(mu, np.ones(8, np.float32))
    assert m.tolist() == [0, 2, 0, 2, -2, 32767, -32768, 0]


@pytest.mark.parametrize("l", [0, 1, 10, 30, 45, 63])
def test_cdf_table_invariants(l):
    t = O.scale_table()
    T = O.cdf_T(l)
    assert T == max(1, math.ceil(7 * float(t[l])))
    f = O.cdf_freq(l).astype(np.int64)
    assert len(f) == 2 * T + 2
    assert f.sum() == 1 << 16 and f.min() >= 1
    # symmetric around zero, peak at zero
    assert np.array_equal(f[:T], f[T + 1:2 * T + 1][::-1])
    assert f[T] == f[:2 * T + 1].max()
    # close to the quantised Gaussian: table cost within the quantisation slack
    sg = float(t[l])
    pmf = np.array([O.likelihood(s, 0.0, sg) for s in range(-T, T + 1)])
    q = f[:2 * T + 1] / 65536.0
    assert np.all(np.abs(q - pmf) <= (2 * T + 3) / 65536.0 + 1e-12)
    # every slot gets at least pmf (1 - n / 2^16) of the range, so the coding
    # loss against the exact pmf is at most -log2(1 - n / 2^16)
    assert np.all(q >= pmf * (1 - (2 * T + 2) / 65536.0) - 1e-15)
    kl = float(np.sum(pmf * np.log2(np.maximum(pmf, 1e-300) / q)))
    assert kl <= -math.log2(1 - (2 * T + 2) / 65536.0)


@pytest.mark.parametrize("l", [0, 1, 10, 30, 45, 63])
def test_cdf_table_closed_form(l):
    """Every slot's frequency from its definition, evaluated through the
    normal distribution function rather than erfc: slot s in -T..T gets
    1 + floor(P(s) (2^16 - n)) with P(s) the mass of [s - 1/2, s + 1/2]
    under N(0, sigma^2), the escape slot the same of P(|s| > T) (both tails),
    and slot 0 the remainder to 2^16.  Where P (2^16 - n) lies within 1e-6 of
    an integer the two evaluations may round apart by one."""
    from scipy.special import ndtr
    t = O.scale_table()
    sg, T = float(t[l]), O.cdf_T(l)
    n = 2 * T + 2
    f = O.cdf_freq(l).astype(np.int64)
    s = np.arange(-T, T + 1, dtype=np.float64)
    p = np.append(ndtr((s + 0.5) / sg) - ndtr((s - 0.5) / sg), 2.0 * ndtr(-(T + 0.5) / sg))
    x = p * (65536 - n)
    want = 1 + np.floor(x).astype(np.int64)
    near = np.abs(x - np.rint(x)) < 1e-6
    rest = np.ones(n, bool)
    rest[T] = False                                  # slot 0 takes the remainder
    assert np.array_equal(f[rest & ~near], want[rest & ~near])
    assert np.all(np.abs(f[rest & near] - want[rest & near]) <= 1)
    assert f[T] == 65536 - f[rest].sum()


# ----------------------------------------------------------- rANS

def _coder_case(c, rng, scale=1.0):
    HW = c.H * c.W
    idx = rng.integers(0, 64, size=(c.H, c.W, c.C)).astype(np.uint8)
    m = rng.integers(-50, 50, size=(c.H, c.W, c.C)).astype(np.int32)
    t = O.scale_table()
    y = np.rint(m + rng.standard_normal((c.H, c.W, c.C)) * t[idx] * scale)
    return np.clip(y, -32767, 32767).astype(np.int16), idx, m


@pytest.mark.parametrize("sched", [0, 1])
def test_rans_round_trip_random(sched):
    c = synth.config("tiny")
    rng = np.random.default_rng(5)
    y, idx, m = _coder_case(c, rng, scale=1.5)       # 1.5 sigma: some escapes
    bs = O.rans_encode(c, sched, y, idx, m)
    ok, yd = O.rans_decode(c, sched, idx, m, bs)
    assert ok and np.array_equal(yd, y)


def test_rans_all_escape_all_zero_single_symbol():
    c = synth.config("tiny")
    rng = np.random.default_rng(6)
    idx = np.zeros((c.H, c.W, c.C), np.uint8)
    m = np.zeros((c.H, c.W, c.C), np.int32)
    # every symbol far outside the support (T = 1 at idx 0), both signs, extremes
    y = rng.choice([-32767, -200, -3, 3, 200, 32767], size=(c.H, c.W, c.C)).astype(np.int16)
    mm = m.copy(); mm[0, 0, 0] = -32768; mm[0, 0, 1] = 32767
    for yy, m_ in ((y, m), (y, mm), (np.zeros_like(y), m)):
        bs = O.rans_encode(c, 0, yy, idx, m_)
        ok, yd = O.rans_decode(c, 0, idx, m_, bs)
        assert ok and np.array_equal(yd, yy)
    one = c.with_grid(1, 1)
    yy = np.array([[[7] * c.C]], np.int16)
    bs = O.rans_encode(one, 0, yy, idx[:1, :1], m[:1, :1])
    ok, yd = O.rans_decode(one, 0, idx[:1, :1], m[:1, :1], bs)
    assert ok and np.array_equal(yd, yy)


def test_rans_size_bound():
    c = synth.config("tiny").with_grid(16, 24)
    rng = np.random.default_rng(8)
    y, idx, m = _coder_case(c, rng)
    bs = O.rans_encode(c, 0, y, idx, m)
    bits = 0.0
    for a in np.ndindex(y.shape):
        l, T = int(idx[a]), O.cdf_T(int(idx[a]))
        f = O.cdf_freq(l)
        s = int(y[a]) - int(m[a])
        slot = s + T if -T <= s <= T else 2 * T + 1
        bits += -math.log2(f[slot] / 65536.0) + (32 if slot == 2 * T + 1 else 0)
    hdr = 16 + 4 * (c.C + 1)
    # per stream: 32 states, at most one unused word per lane, one pad word
    slack = c.C * (32 * 32 + 32 * 16 + 16)
    assert (len(bs) - hdr) * 8 <= bits + slack


@pytest.mark.parametrize("name,sched,grid", [("tiny", 0, None), ("tiny", 1, None), ("tiny_cyc", 0, None),
                                            ("tiny", 0, (3, 37)), ("tiny", 0, (1, 1))])
def test_rans_container_read_by_an_independent_reader(name, sched, grid):
    """The oracle's containers read back by a plain reader written from the
    format alone (tests/rans_ref.py: header, offsets, lane states, word
    order, slots, escape digits, schedule order, final states): random
    symbols with escapes and int16 extremes, 2i+j, raster and cyclic orders,
    a ragged and a 1 x 1 grid."""
    import rans_ref
    c = synth.config(name)
    if grid:
        c = c.with_grid(*grid)
    rng = np.random.default_rng(31 + sched)
    y, idx, m = _coder_case(c, rng, scale=1.5)
    y[..., 0] = rng.choice([-32767, 32767], size=y.shape[:2])
    idx[..., 0] = 0
    m[..., 0] = 0
    bs = O.rans_encode(c, sched, y, idx, m)
    freqs = {l: O.cdf_freq(l).astype(np.int64) for l in range(64)}
    HW = c.H * c.W
    yd = rans_ref.decode(bs, c.H, c.W, c.C, sched, c.mask, idx.reshape(HW, c.C), m.reshape(HW, c.C), freqs)
    assert np.array_equal(yd.reshape(y.shape), y.astype(np.int64))


def test_zhat_container_read_by_an_independent_reader():
    """The z-hat container (raster order over the hyperprior grid, channel
    ch coded with its factorized-prior table about mean 0) read back by the
    same plain reader, with escapes past the tables' +-31 support."""
    import rans_ref
    c = synth.config("tiny_hp")
    w = synth.weights(c).astype(np.float64)
    rng = np.random.default_rng(41)
    zh = rng.integers(-6, 7, size=(c.Hh, c.Wh, c.Ch)).astype(np.int16)
    zh[0, 0, :4] = [40, -40, 32767, -32768]
    bs = O.hyper_encode(c, w, zh)
    HW = c.Hh * c.Wh
    freqs = {ch: O.prior_freq(c, w, ch).astype(np.int64) for ch in range(c.Ch)}
    idx = np.tile(np.arange(c.Ch), (HW, 1))
    zd = rans_ref.decode(bs, c.Hh, c.Wh, c.Ch, 1, 0, idx, np.zeros((HW, c.Ch), np.int64), freqs)
    assert np.array_equal(zd.reshape(zh.shape), zh.astype(np.int64))


def test_rans_detects_corruption():
    c = synth.config("tiny")
    rng = np.random.default_rng(9)
    y, idx, m = _coder_case(c, rng)
    bs = bytearray(O.rans_encode(c, 0, y, idx, m))
    ok, _ = O.rans_decode(c, 0, idx, m, bytes(bs[:-10]))       # truncated
    assert not ok
    bad = bytearray(bs); bad[0] ^= 1                            # magic
    assert not O.rans_decode(c, 0, idx, m, bytes(bad))[0]
    bad = bytearray(bs); bad[6] = 1                             # wrong schedule
    assert not O.rans_decode(c, 0, idx, m, bytes(bad))[0]
    hdr = 16 + 4 * (c.C + 1)
    flips = 0
    for pos in rng.integers(hdr + 128, len(bs), size=20):
        bad = bytearray(bs); bad[pos] ^= 0x5A
        ok, yd = O.rans_decode(c, 0, idx, m, bytes(bad))
        flips += (not ok) or (not np.array_equal(yd, y))
    assert flips == 20


def test_rans_decoded_latent_outside_int16_is_an_error():
    """A container decoded against means other than the encoder's can give a
    latent m + s outside int16: that is reported as corrupt, not wrapped.
    y = +-32767 coded at mean 0; decoding with the means moved 10 outward
    leaves the int16 range at exactly those positions, while moving them 10
    inward gives y -+ 10 and no error."""
    c = synth.config("tiny").with_grid(2, 3)
    y = np.zeros((c.H, c.W, c.C), np.int16)
    y[0, 0, 0], y[1, 2, c.C - 1] = 32767, -32767
    idx = np.full(y.shape, 10, np.uint8)
    m = np.zeros(y.shape, np.int32)
    bs = O.rans_encode(c, 0, y, idx, m)
    assert O.rans_decode(c, 0, idx, m, bs)[0]
    out = m.copy()
    out[0, 0, 0], out[1, 2, c.C - 1] = 10, -10
    assert not O.rans_decode(c, 0, idx, out, bs)[0]
    ok, yd = O.rans_decode(c, 0, idx, -out, bs)
    assert ok and yd[0, 0, 0] == 32757 and yd[1, 2, c.C - 1] == -32757


def test_encode_decode_round_trip_through_the_model():
    for nm, nf in (("tiny", 1), ("tiny_p", 3), ("tiny_ct", 1), ("tiny_cyc_ct", 1), ("tiny_p_ct", 2)):
        c = synth.config(nm)
        w = synth.weights(c)
        fr = synth.frames(c, nf, seed=12)
        bs, mu, sg = O.encode_frames(c, w, fr.y, fr.z)
        yd, mud, sgd = O.decode_frames(c, w, bs, fr.z)
        assert np.array_equal(yd, fr.y)
        assert np.array_equal(mu, mud) and np.array_equal(sg, sgd)


# ----------------------------------------------------------- data generator

def test_generator_statistics():
    c = synth.config("i1080")
    rng = np.random.Generator(np.random.PCG64(0))
    x = synth.ar1_field(rng, 68, 120, 64, 0.8)
    assert abs(x.var() - 1.0) < 0.05
    r_h = np.mean(x[:, 1:] * x[:, :-1]); r_v = np.mean(x[1:] * x[:-1])
    assert abs(r_h - 0.8) < 0.03 and abs(r_v - 0.8) < 0.03
    assert abs(np.mean(x[1:, 1:] * x[:-1, :-1]) - 0.64) < 0.04
    fr = synth.frames(c.with_grid(34, 60), 2, seed=1)
    assert fr.y.dtype == np.int16 and fr.y.shape == (2, 34, 60, 192)
    ls = np.log(fr.sigma).ravel()
    assert abs(ls.min() - math.log(0.1)) < 0.05 and abs(ls.max() - math.log(8)) < 0.05
    hist, _ = np.histogram(ls, bins=4)
    assert hist.min() > 0.7 * hist.mean()            # log-uniform
    a, b = fr.y[0].astype(float) / fr.sigma[..., None], fr.y[1].astype(float) / fr.sigma[..., None]
    big = fr.sigma > 3
    assert abs(np.corrcoef(a[big].ravel(), b[big].ravel())[0, 1] - 0.9) < 0.05
