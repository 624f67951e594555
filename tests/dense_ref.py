"""Dense-mask NumPy formulation of the P-SWA context model, for tiny frames.

Test helper used to pin the oracle.  It follows the same reading of the
paper as the oracle (Sec. 3.1 block structure, Sec. 3.2 / Fig. 2 masks) but
is written as a textbook masked transformer: every layer runs full
[HW x HW] attention with a boolean mask matrix and a bias matrix, instead of
the oracle's clipped per-position window key lists.  Window clipping, key
order, bias offsets and the weight packing order (taken here from the
synthetic-input module's tensor list, not from the oracle's own layout code)
are therefore computed a second, different way.  Only for small H*W.
"""
from __future__ import annotations

import numpy as np

from paper_2605_20977_gb300 import synth


def split_weights(c: synth.ModelConfig, w: np.ndarray) -> dict:
    out, o = {}, 0
    for t in synth.weight_spec(c):
        n = int(np.prod(t.shape))
        out[t.name] = np.asarray(w[o:o + n], np.float64).reshape(t.shape)
        o += n
    assert o == w.size
    return out


def grid_masks(c: synth.ModelConfig):
    """Boolean [HW, HW] matrices indexed [p, q]: window, A (accumulator),
    S (spatial self-attention); and the window offset index of q - p."""
    H, W, w = c.H, c.W, (c.k - 1) // 2
    ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    ii, jj = ii.ravel(), jj.ravel()
    if c.mask == 0:
        lab = 2 * ii + jj
    else:
        lab = (ii % 4 + jj % 4) % 4
    rho = ii * W + jj
    di = ii[None, :] - ii[:, None]
    dj = jj[None, :] - jj[:, None]
    win = (np.abs(di) <= w) & (np.abs(dj) <= w)
    before = rho[None, :] < rho[:, None]
    lq, lp = lab[None, :], lab[:, None]
    A = win & (lq < lp)
    S = win & (lq <= lp)
    if c.mask == 0:
        A &= before
        S &= before | (rho[None, :] == rho[:, None])
    off = np.where(win, (di + w) * c.k + (dj + w), 0)
    return win, A, S, off


def rms(x, g):
    return x / np.sqrt(np.mean(x * x, axis=-1, keepdims=True) + 1e-6) * g


def silu(x):
    return x / (1.0 + np.exp(-x))


def attention(Q, K, V, M, B, nh):
    """Q [P, d], K/V [N, d], M [P, N] bool, B [nh, P, N].  Rows with no
    visible key give 0."""
    P, d = Q.shape
    dh = d // nh
    out = np.zeros((P, d))
    for h in range(nh):
        sl = slice(h * dh, (h + 1) * dh)
        s = Q[:, sl] @ K[:, sl].T / np.sqrt(dh) + B[h]
        s = np.where(M, s, -np.inf)
        has = M.any(axis=1)
        mx = np.where(has, s.max(axis=1, initial=-np.inf), 0.0)
        e = np.where(M, np.exp(s - mx[:, None]), 0.0)
        z = e.sum(axis=1)
        pr = np.divide(e, z[:, None], out=np.zeros_like(e), where=has[:, None])
        out[:, sl] = pr @ V[:, sl]
    return out


def ffn(x, Wg, Wu, Wd):
    return (silu(x @ Wg) * (x @ Wu)) @ Wd


def conv3(x, W, b, stride=1):
    """3x3 correlation with zero padding 1: x [h][w][Ci], W [3][3][Ci][Co]
    -> [ceil(h/stride)][ceil(w/stride)][Co], as nine shifted views."""
    h, w_, _ = x.shape
    ho, wo = -(-h // stride), -(-w_ // stride)
    xp = np.pad(x, ((1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(b, (ho, wo, W.shape[3])).copy()
    for di in range(3):
        for dj in range(3):
            v = xp[di:di + stride * (ho - 1) + 1:stride, dj:dj + stride * (wo - 1) + 1:stride]
            out += np.tensordot(v, W[di, dj], axes=([2], [0]))
    return out


def shuffle2(u):
    """[h][w][4C] -> [2h][2w][C], channel (2a + b) C + c to sub-position (a, b)."""
    h, w_, c4 = u.shape
    return u.reshape(h, w_, 2, 2, c4 // 4).transpose(0, 2, 1, 3, 4).reshape(2 * h, 2 * w_, c4 // 4)


def lrelu(x):
    return np.where(x >= 0, x, 0.01 * x)


def rb_down(P, pre, x):
    a = lrelu(conv3(x, P[pre + "Wa"], P[pre + "ba"], 2))
    return conv3(a, P[pre + "Wb"], P[pre + "bb"]) + (x[::2, ::2] @ P[pre + "Ws"] + P[pre + "bs"])


def rb_up(P, pre, x):
    a = lrelu(shuffle2(conv3(x, P[pre + "Wa"], P[pre + "ba"])))
    return conv3(a, P[pre + "Wb"], P[pre + "bb"]) + shuffle2(conv3(x, P[pre + "Ws"], P[pre + "bs"]))


def run(c: synth.ModelConfig, w: np.ndarray, y: np.ndarray, z: np.ndarray, with_eps: bool = False,
        with_z: bool = False):
    """(mu, sigma) [nf, H, W, C] for a sequence, by the masked parallel pass;
    with with_eps also the LRP Transformer's residual eps of every frame
    (full [HW x HW] attention under the unmasked window mask); with with_z
    (a convolutional hyperprior model) also the unrounded analysis output z
    of every frame, from that frame's Spatial Module 1 output."""
    P = split_weights(c, w)
    H, W, C, d, nh = c.H, c.W, c.C, c.d, c.nh
    HW = H * W
    win, A, S, off = grid_masks(c)
    nf = y.shape[0]

    def bias_of(tab):                     # tab [nh, k, k] -> [nh, HW, HW]
        return tab.reshape(nh, -1)[:, off]

    # Context Transformer over all frames (time-causal, spatially unmasked).
    ctx_out = []
    if c.temporal:
        g = []
        for f in range(nf):
            if f == 0:
                g.append(np.tile(P["pad"], (HW, 1)))
            else:
                g.append((y[f - 1].reshape(HW, C) * P["gamma_c"]) @ P["W_c"] + P["b_c"])
        for l in range(c.Lc):
            pre = f"ctx{l}."
            n = [rms(gf, P[pre + "g_attn"]) for gf in g]
            Q = [a @ P[pre + "Wq"] for a in n]
            K = [a @ P[pre + "Wk"] for a in n]
            V = [a @ P[pre + "Wv"] for a in n]
            tb = P[pre + "bias"]                          # [nh, Tf, k, k]
            new = []
            for f in range(nf):
                fs = list(range(max(0, f - c.Tf + 1), f + 1))
                Kc = np.concatenate([K[ff] for ff in fs])
                Vc = np.concatenate([V[ff] for ff in fs])
                M = np.concatenate([win for _ in fs], axis=1)
                B = np.concatenate([tb[:, f - ff].reshape(nh, -1)[:, off] for ff in fs], axis=2)
                a = g[f] + attention(Q[f], Kc, Vc, M, B, nh) @ P[pre + "Wo"]
                a = a + ffn(rms(a, P[pre + "g_ffn"]), P[pre + "Wg"], P[pre + "Wu"], P[pre + "Wd"])
                new.append(a)
            g = new
        ctx_out = [rms(gf, P["g_ctx"]) for gf in g]

    def block(pre, x, M, f):
        n = rms(x, P[pre + "g_attn"])
        x = x + attention(n @ P[pre + "Wq"], n @ P[pre + "Wk"], n @ P[pre + "Wv"], M,
                          bias_of(P[pre + "bias"]), nh) @ P[pre + "Wo"]
        if c.temporal:
            fs = list(range(max(0, f - c.Tf + 1), f + 1))
            Kc = np.concatenate([ctx_out[ff] @ P[pre + "Wxk"] for ff in fs])
            Vc = np.concatenate([ctx_out[ff] @ P[pre + "Wxv"] for ff in fs])
            Mc = np.concatenate([win for _ in fs], axis=1)
            Bc = np.concatenate([P[pre + "xbias"][:, f - ff].reshape(nh, -1)[:, off] for ff in fs], axis=2)
            qx = rms(x, P[pre + "g_x"]) @ P[pre + "Wxq"]
            x = x + attention(qx, Kc, Vc, Mc, Bc, nh) @ P[pre + "Wxo"]
        return x + ffn(rms(x, P[pre + "g_ffn"]), P[pre + "Wg"], P[pre + "Wu"], P[pre + "Wd"])

    mus, sigs, epss, zs = [], [], [], []
    nb = int(round(np.log2(c.r)))
    LK = [[] for _ in range(c.Llrp)]       # LRP keys / values of every coded frame, per block
    LV = [[] for _ in range(c.Llrp)]
    for f in range(nf):
        ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        if c.hp:
            xh = z[f].astype(np.float64) * P["gamma_z"]
            for b in range(nb):
                xh = rb_up(P, f"hp.u{b}.", xh)
            eh = xh[:H, :W].reshape(HW, d)
        else:
            zz = z[f][ii // c.r, jj // c.r].reshape(HW, c.Ch) * P["gamma_z"]
            sub = ((ii % c.r) * c.r + (jj % c.r)).ravel()
            eh = np.einsum("pc,pcd->pd", zz, P["W_hp"][sub]) + P["b_hp"]
        x1 = (y[f].reshape(HW, C) * P["gamma_in"]) @ P["W_in"] + P["b_in"]
        for l in range(c.L):
            x1 = block(f"sm1.{l}.", x1, S, f)
        if with_z:
            xa = rms(x1, P["hp.g_za"]).reshape(H, W, d)
            for b in range(nb):
                xa = rb_down(P, f"hp.d{b}.", xa)
            zs.append(xa)
        m = rms(x1, P["acc.g_kv"])
        qa = rms(eh, P["acc.g_q"]) @ P["acc.Wq"]
        x2 = eh + attention(qa, m @ P["acc.Wk"], m @ P["acc.Wv"], A, bias_of(P["acc.bias"]), nh) @ P["acc.Wo"]
        x2 = x2 + ffn(rms(x2, P["acc.g_ffn"]), P["acc.Wg"], P["acc.Wu"], P["acc.Wd"])
        for l in range(c.L):
            x2 = block(f"sm2.{l}.", x2, S, f)
        if c.Nc:
            # Channel Transformer over all positions at once: groups as
            # column blocks, the mask as a Kronecker block pattern
            G, dg, Cg = c.Nc, c.dc // c.Nc, C // c.Nc
            grms = lambda x, g: np.concatenate([rms(x[:, j * dg:(j + 1) * dg], g[j * dg:(j + 1) * dg])
                                                for j in range(G)], axis=1)
            yl = y[f].reshape(HW, C) * P["ct.gamma_y"]
            shifted = np.concatenate([np.zeros((HW, dg))] +
                                     [yl[:, (j - 1) * Cg:j * Cg] @ P["ct.E"][j - 1] for j in range(1, G)], axis=1)
            h = rms(x2, P["ct.g_in"]) @ P["ct.W_in"] + P["ct.b_in"] + shifted
            keep = np.kron(np.triu(np.ones((G, G))), np.ones((dg, dg)))      # [in group, out group]: in <= out
            for l in range(c.Lct):
                pre = f"ct{l}."
                h = h + grms(h, P[pre + "g_mix"]) @ (P[pre + "M"] * keep)
                a = grms(h, P[pre + "g_ffn"])
                h = h + np.concatenate([ffn(a[:, j * dg:(j + 1) * dg], P[pre + "Wg"][j], P[pre + "Wu"][j],
                                            P[pre + "Wd"][j]) for j in range(G)], axis=1)
            x2 = h                                   # the heads' input (and the LRP's representation)
            n = grms(h, P["g_head"])
            hm = [silu(n[:, j * dg:(j + 1) * dg] @ P["W1m"][j] + P["b1m"][j * dg:(j + 1) * dg]) @ P["W2m"][j]
                  for j in range(G)]
            hs = [silu(n[:, j * dg:(j + 1) * dg] @ P["W1s"][j] + P["b1s"][j * dg:(j + 1) * dg]) @ P["W2s"][j]
                  for j in range(G)]
            mu = P["gamma_mu"] * np.concatenate(hm, axis=1) + P["beta_mu"]
            s = P["gamma_sig"] * np.concatenate(hs, axis=1) + P["beta_sig"]
        else:
            n = rms(x2, P["g_head"])
            mu = P["gamma_mu"] * (silu(n @ P["W1m"] + P["b1m"]) @ P["W2m"]) + P["beta_mu"]
            s = P["gamma_sig"] * (silu(n @ P["W1s"] + P["b1s"]) @ P["W2s"]) + P["beta_sig"]
        sig = np.exp(np.clip(s, np.log(0.11), np.log(256.0)))
        mus.append(mu.reshape(H, W, C)); sigs.append(sig.reshape(H, W, C))
        if with_eps:
            u = (rms(x2, P["lrp.g_rep"]) @ P["lrp.W_rep"] + (y[f].reshape(HW, C) * P["lrp.gamma_y"]) @ P["lrp.W_y"]
                 + P["lrp.b_in"])
            for l in range(c.Llrp):
                pre = f"lrp{l}."
                n = rms(u, P[pre + "g_attn"])
                LK[l].append(n @ P[pre + "Wk"])
                LV[l].append(n @ P[pre + "Wv"])
                # time-causal for the temporal model: the windows of the
                # current and Tf - 1 previous frames, bias by frame age
                fs = list(range(max(0, f - c.Tf + 1), f + 1)) if c.temporal else [f]
                tb = P[pre + "bias"].reshape(nh, -1, c.k * c.k)
                Kc = np.concatenate([LK[l][ff] for ff in fs])
                Vc = np.concatenate([LV[l][ff] for ff in fs])
                M = np.concatenate([win for _ in fs], axis=1)
                B = np.concatenate([tb[:, f - ff][:, off] for ff in fs], axis=2)
                u = u + attention(n @ P[pre + "Wq"], Kc, Vc, M, B, nh) @ P[pre + "Wo"]
                u = u + ffn(rms(u, P[pre + "g_ffn"]), P[pre + "Wg"], P[pre + "Wu"], P[pre + "Wd"])
            epss.append((rms(u, P["lrp.g_out"]) @ P["lrp.W_eps"] + P["lrp.b_eps"]).reshape(H, W, C))
    out = (np.stack(mus), np.stack(sigs))
    if with_eps:
        out = out + (np.stack(epss),)
    if with_z:
        out = out + (np.stack(zs),)
    return out
