"""An independent reader of the coder's container, written from its format
alone, to pin the bytes the oracle's encoder writes (test code, plain
Python loops, small frames only).

The format (little endian): a 16-byte header -- u32 magic "PSW1", u16
version 1, u16 schedule, u16 H, u16 W, u16 C, u16 0 -- then u32 offsets of
the C channel streams and of the end.  A channel stream holds the 32 lane
states (u32 each), then 16-bit renormalisation words in the order the
decoder reads them, then one zero word if needed to end on a multiple of 4
bytes.  Symbol k of a channel (positions in schedule order: raster order, or
the positions of each step label in raster order) is on lane k mod 32.  A
symbol's slot is the last one whose cumulative frequency is at most the low
16 bits of the lane's state; the state becomes f (x >> 16) + (x & 0xFFFF) -
cum, then takes one word if it fell below 2^16.  Slots 0..2T are the values
-T..T about the rounded mean; slot 2T + 1 is the escape, after which two
16-bit digits d0 (low) then d1 of v = 2 (|s| - T - 1) + (s < 0) are taken
from the low half of the state, each followed by one word.  Every lane ends
at 2^16 and every stream is read to its end.
"""
import numpy as np

MAGIC = 0x31575350          # "PSW1"
LOW = 1 << 16


def schedule_order(H, W, sched, mask):
    """Positions in coding order: raster (sched 1), else by step label
    (2i + j, or ((i mod 4) + (j mod 4)) mod 4 for the cyclic mask) and raster
    order within a label."""
    if sched == 1:
        return list(range(H * W))
    if mask == 1:
        label = lambda i, j: ((i % 4) + (j % 4)) % 4
    else:
        label = lambda i, j: 2 * i + j
    return sorted(range(H * W), key=lambda p: (label(p // W, p % W), p))


def decode(buf, H, W, C, sched, mask, idx, m, freqs):
    """Latents [H*W][C] from a container; idx, m: [H*W][C] table index and
    rounded mean of each symbol; freqs[l]: table l's slot frequencies (2T+2
    of them, the last the escape).  Raises AssertionError on any departure
    from the format."""
    b = bytes(buf)
    u16 = lambda o: b[o] | (b[o + 1] << 8)
    u32 = lambda o: u16(o) | (u16(o + 2) << 16)
    assert u32(0) == MAGIC and u16(4) == 1 and u16(6) == sched
    assert (u16(8), u16(10), u16(12), u16(14)) == (H, W, C, 0)
    offs = [u32(16 + 4 * c) for c in range(C + 1)]
    assert offs[0] == 16 + 4 * (C + 1) and offs[-1] == len(b)
    cums = {}
    order = schedule_order(H, W, sched, mask)
    y = np.zeros((H * W, C), np.int64)
    for c in range(C):
        a0, a1 = offs[c], offs[c + 1]
        x = [u32(a0 + 4 * l) for l in range(32)]
        p = a0 + 128
        for k, pos in enumerate(order):
            lane, l = k % 32, int(idx[pos][c])
            f = freqs[l]
            if l not in cums:
                cums[l] = np.concatenate([[0], np.cumsum(f)]).astype(np.int64)
            cum, T = cums[l], (len(f) - 2) // 2
            v = x[lane] & 0xFFFF
            s = int(np.searchsorted(cum, v, side="right")) - 1
            x[lane] = int(f[s]) * (x[lane] >> 16) + v - int(cum[s])
            if x[lane] < LOW:
                assert p + 2 <= a1
                x[lane] = (x[lane] << 16) | u16(p)
                p += 2
            if s == 2 * T + 1:
                d = []
                for _ in range(2):
                    d.append(x[lane] & 0xFFFF)
                    assert p + 2 <= a1
                    x[lane] = (x[lane] & 0xFFFF0000) | u16(p)
                    p += 2
                vv = d[0] | (d[1] << 16)
                mag = T + 1 + (vv >> 1)
                sv = -mag if vv & 1 else mag
            else:
                sv = s - T
            y[pos][c] = int(m[pos][c]) + sv
        assert all(xl == LOW for xl in x)
        assert p == a1 or (p + 2 == a1 and u16(p) == 0)
    return y
