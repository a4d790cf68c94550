"""GPU BC6H encoders (Sec. 5.1 partition selection; the plain two-mode
compressor) against the CPU oracle's double-precision search, by what is
fixed whatever the summation order:
  - the GPU's encoding, read back through the oracle's format decoder, has
    the squared error the GPU reports;
  - every index is the best one for its endpoints;
  - the GPU's decoded error is at most the oracle's (the GPU refines the
    winner of the same search), up to single-precision error sums;
  - blocks that are themselves encodings are reproduced exactly.
"""
import zlib

import numpy as np
import pytest
import torch

import oracle

pytestmark = pytest.mark.gpu


def _bcf():
    import paper_2311_16121_b300 as bcf

    bcf.lib()
    return bcf


def _level_texels(rng, W, kind):
    if kind == "noise":
        return rng.random((W, W, 3), dtype=np.float32)
    if kind == "smooth":
        y, x = np.meshgrid(np.arange(W), np.arange(W), indexing="ij")
        f = [np.sin(x * a + y * b + c) for a, b, c in rng.uniform(0.05, 0.6, (3, 3))]
        return (0.5 + 0.4 * np.stack(f, -1)).astype(np.float32)
    if kind == "wide":  # values across the half range, zeros, negatives, above the range
        v = np.exp(rng.uniform(-12, 11.5, (W, W, 3))).astype(np.float32)
        v[rng.random((W, W, 3)) < 0.05] = 0.0
        v[rng.random((W, W, 3)) < 0.05] *= -1.0
        v[rng.random((W, W, 3)) < 0.01] = 70000.0
        return v
    if kind == "exact":  # every block a mode-10 lattice block (the encoder reproduces them exactly)
        out = np.zeros((W, W, 3), np.float32)
        for by in range(W // 4):
            for bx in range(W // 4):
                k = int(rng.integers(0, 32))
                while True:  # both segment ends used in each region, ends apart: the line fit sees the segment
                    e = rng.integers(0, 64, (4, 3))
                    if all(np.abs(e[2 * r] - e[2 * r + 1]).max() >= 8 for r in range(2)):
                        break
                idx = rng.integers(0, 8, 16)
                for r in range(2):
                    ts = [t for t in range(16) if oracle.bc6h_partition_region(k, t) == r]
                    i0, i1 = rng.choice(ts, 2, replace=False)
                    idx[i0], idx[i1] = 0, 7
                p = np.concatenate([e.reshape(-1), idx / 7.0])
                mode, tex = oracle.bc6h_decode_block(oracle.train_export_block(p, k))
                vals = np.array([[oracle.half_to_double(int(tex[t, c])) for c in range(3)] for t in range(16)])
                out[4 * by:4 * by + 4, 4 * bx:4 * bx + 4] = vals.reshape(4, 4, 3)
        return out
    if kind == "constant":
        return np.full((W, W, 3), rng.random(3, dtype=np.float32), np.float32)
    raise ValueError(kind)


def _texture(rng, res, levels, kinds):
    return np.concatenate([_level_texels(rng, res >> l, kinds[l % len(kinds)]).reshape(-1) for l in range(levels)])


def _block_targets(tex, res, levels, stride=3):
    """The input texels of every block, [blocks][16][3] float32 in the encoders' block order."""
    out, off = [], 0
    for l in range(levels):
        W = res >> l
        img = tex[off:off + W * W * stride].reshape(W, W, stride)[:, :, :3]
        out.append(img.reshape(W // 4, 4, W // 4, 4, 3).transpose(0, 2, 1, 3, 4).reshape(-1, 16, 3))
        off += W * W * stride
    return np.concatenate(out)


def _values(blk):
    _, tex = oracle.bc6h_decode_block(blk)
    return tex.view(np.float16).astype(np.float64)


def _index_errors_mode10(p28, k, target):
    """[8][16] squared error of every texel at each 3-bit index for the record's endpoints (each plane is the
    record with all positions at one index, exported and read by the oracle's format decoder)."""
    out = np.zeros((8, 16))
    for i in range(8):
        q = p28.copy()
        q[12:] = i / 7.0
        out[i] = ((_values(oracle.train_export_block(q, k)) - target) ** 2).sum(axis=1)
    return out


def _check_mode10(p32, part, err, targets, ref_err, what):
    """Validity of the GPU's mode-10 encodings, and its error against the oracle's search: returns how many
    blocks the GPU encodes strictly better."""
    assert not p32[:, [6, 7, 14, 15]].any()
    better = 0
    for b in range(p32.shape[0]):
        p28 = np.concatenate([p32[b, 0:6], p32[b, 8:14], p32[b, 16:32]]).astype(np.float64)
        k = int(part[b])
        assert 0 <= k < 32 and np.array_equal(p28[:12], np.round(p28[:12])) and (0 <= p28[:12]).all() and \
            (p28[:12] <= 63).all(), (what, b)
        idx = np.rint(p28[12:] * 7).astype(int)
        assert np.allclose(p28[12:], idx / 7.0, rtol=0, atol=1e-7), (what, b)
        tgt = targets[b].astype(np.float64)
        e_idx = _index_errors_mode10(p28, k, tgt)
        chosen = e_idx[idx, np.arange(16)]
        assert (chosen <= e_idx.min(axis=0) * (1 + 1e-6) + 1e-12).all(), (what, b, "index not optimal")
        dec = chosen.sum()
        assert err[b] == pytest.approx(dec, rel=1e-5, abs=1e-9), (what, b, err[b], dec)
        assert dec <= ref_err[b] * (1 + 1e-5) + 1e-12, (what, b, dec, ref_err[b])
        better += dec < ref_err[b] * (1 - 1e-5)
    return better


def _compare(bcf, tex, res, levels):
    p, part, err = bcf.encode_mode10(torch.from_numpy(tex).cuda(), res, levels)
    p, part, err = p.cpu().numpy(), part.cpu().numpy(), err.cpu().numpy()
    _, _, rerr = oracle.encode_mode10_texture(tex, res, levels)
    better = _check_mode10(p, part, err, _block_targets(tex, res, levels), rerr, (res, levels))
    print(f"{res}^2 x {levels} levels: {p.shape[0]} blocks, GPU error below the oracle's on {better}")
    return part, err


@pytest.mark.parametrize("kinds", [("noise",), ("smooth", "wide"), ("exact", "constant", "noise")])
def test_encoder_is_valid_and_at_least_as_good_as_the_oracle(kinds):
    """bcf_encode_mode10 on noise, smooth, wide-range, exactly encodable and constant levels: valid records,
    optimal indices, the reported error, and an error at most the oracle's search's."""
    bcf = _bcf()
    rng = np.random.default_rng(zlib.crc32("/".join(kinds).encode()))
    res, levels = 64, 5
    tex = _texture(rng, res, levels, kinds)
    part, err = _compare(bcf, tex, res, levels)
    if kinds[0] == "exact":  # level 0 is all exact blocks: zero error everywhere there
        assert not err[:256].any()


def test_encoder_texel_stride_4():
    """The unconstrained training features' layout ([texels][4]) encodes like the packed RGB one."""
    bcf = _bcf()
    rng = np.random.default_rng(9)
    tex3 = _texture(rng, 32, 4, ("smooth", "noise"))
    tex4 = np.concatenate([tex3.reshape(-1, 3), np.full((tex3.size // 3, 1), 7.0, np.float32)], axis=1)
    a = bcf.encode_mode10(torch.from_numpy(tex3).cuda(), 32, 4)
    b = bcf.encode_mode10(torch.from_numpy(tex4.reshape(-1)).cuda(), 32, 4, texel_stride=4)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_encoder_edge_sizes():
    bcf = _bcf()
    rng = np.random.default_rng(7)
    for res, levels in ((4, 1), (8, 1), (8, 2), (16, 3)):
        _compare(bcf, _texture(rng, res, levels, ("noise", "smooth")), res, levels)


def test_encoder_full_size_sampled():
    """1024^2 with 9 levels (87,381 blocks): 600 sampled blocks checked as in the small cases."""
    bcf = _bcf()
    rng = np.random.default_rng(8)
    res, levels = 1024, 9
    tex = _texture(rng, res, levels, ("smooth", "noise"))
    p, part, err = (a.cpu().numpy() for a in bcf.encode_mode10(torch.from_numpy(tex).cuda(), res, levels))
    nb = oracle.texture_blocks(res, levels)
    assert p.shape == (nb, 32)
    # level offsets of the blocks and of the texels
    boffs, toffs, b, t = [], [], 0, 0
    for l in range(levels):
        W = res >> l
        boffs.append(b)
        toffs.append(t)
        b += (W // 4) ** 2
        t += W * W * 3
    pick = np.sort(rng.choice(nb, 600, replace=False))
    targets, rerr = [], []
    for bi in pick:
        l = max(i for i in range(levels) if boffs[i] <= bi)
        W = res >> l
        by, bx = divmod(int(bi - boffs[l]), W // 4)
        img = tex[toffs[l]:toffs[l] + W * W * 3].reshape(W, W, 3)
        blk = img[4 * by:4 * by + 4, 4 * bx:4 * bx + 4].reshape(16, 3)
        targets.append(blk)
        rerr.append(oracle.encode_mode10_block(blk)[2])
    _check_mode10(p[pick], part[pick], err[pick], np.stack(targets), np.array(rerr), "full size")


def test_encoder_rejects_bad_arguments():
    bcf = _bcf()
    tex = torch.zeros(2 * 64 * 64 * 3, device="cuda")
    with pytest.raises(bcf.BcfError):
        bcf.encode_mode10(tex, 64, 6)  # 64 -> at most 5 levels
    with pytest.raises(bcf.BcfError):
        bcf.encode_mode10(tex, 64, 1, texel_stride=5)
    with pytest.raises(ValueError):
        bcf.encode_mode10(tex[:100], 64, 1)  # too few texels


@pytest.mark.parametrize("is_signed", [False, True])
def test_pack_mode10_matches_oracle_export(is_signed):
    """bcf_pack_mode10 on arbitrary records (codes beyond the clamp range, positions outside [0, 1], anchors
    needing the swap) equals the oracle's export bit for bit; unsigned and signed."""
    bcf = _bcf()
    rng = np.random.default_rng(61 + is_signed)
    nb = 3000
    p28 = np.concatenate([rng.uniform(-40 if is_signed else -5, 68 if not is_signed else 40, (nb, 12)),
                          rng.uniform(-0.2, 1.2, (nb, 16))], axis=1).astype(np.float32)
    p32 = np.zeros((nb, 32), np.float32)
    p32[:, 0:6], p32[:, 8:14], p32[:, 16:32] = p28[:, 0:6], p28[:, 6:12], p28[:, 12:28]
    k = rng.integers(0, 32, nb).astype(np.uint8)
    got = bcf.pack_mode10(torch.from_numpy(p32).cuda(), torch.from_numpy(k).cuda(), is_signed=is_signed)
    got = got.cpu().numpy().reshape(nb, 16)
    ref = np.stack([oracle.train_export_block(p28[i], int(k[i]), is_signed=is_signed) for i in range(nb)])
    np.testing.assert_array_equal(got, ref)


def test_encode_then_pack_is_a_mode10_compressor():
    """encode + pack: every block decodes (bcf_decode_bc6h) to the encoder's reported error, computed here from
    the decoded values against the input texels."""
    bcf = _bcf()
    rng = np.random.default_rng(67)
    res, levels = 32, 3
    tex = _texture(rng, res, levels, ("smooth", "noise"))
    p, part, err = bcf.encode_mode10(torch.from_numpy(tex).cuda(), res, levels)
    blocks = bcf.pack_mode10(p, part)
    off_b, off_t = 0, 0
    for lvl in range(levels):
        W = res >> lvl
        nb = (W // 4) ** 2
        dec = bcf.decode_bc6h(blocks[16 * off_b:16 * (off_b + nb)], W // 4, W // 4).cpu().numpy()
        vals = dec.view(np.float16).astype(np.float32).reshape(W, W, 3)
        src = tex[off_t:off_t + W * W * 3].reshape(W, W, 3)
        sq = ((vals - src) ** 2).reshape(W // 4, 4, W // 4, 4, 3).transpose(0, 2, 1, 3, 4).reshape(nb, 48)
        e = err[off_b:off_b + nb].cpu().numpy()
        np.testing.assert_allclose(sq.astype(np.float64).sum(1), e, rtol=1e-5, atol=1e-9)
        off_b += nb
        off_t += W * W * 3


def _mode11_level(rng, W):
    """Every block a mode-11 lattice block (the compressor reproduces them exactly, in mode 11)."""
    out = np.zeros((W, W, 3), np.float32)
    for by in range(W // 4):
        for bx in range(W // 4):
            while True:
                e = rng.integers(0, 1024, (2, 3))
                if np.abs(e[0] - e[1]).max() >= 64:
                    break
            idx = rng.integers(0, 16, 16)
            idx[0] = rng.integers(0, 8)
            i0, i1 = rng.choice(np.arange(1, 16), 2, replace=False)
            idx[i0], idx[i1] = 0, 15
            blk = oracle.bc6h_encode_fields(11, [int(x) for x in e.reshape(-1)] + [0] * 6, 0, [int(i) for i in idx])
            _, tex = oracle.bc6h_decode_block(blk)
            vals = np.array([[oracle.half_to_double(int(tex[t, c])) for c in range(3)] for t in range(16)])
            out[4 * by:4 * by + 4, 4 * bx:4 * bx + 4] = vals.reshape(4, 4, 3)
    return out


@pytest.mark.parametrize("kinds", [("noise",), ("smooth", "wide"), ("exact", "constant", "mode11")])
def test_compressor_is_valid_and_at_least_as_good_as_the_oracle(kinds):
    """bcf_compress_bc6h: every block is mode 10 or 11, decodes (oracle format decoder) to the reported error, is
    at most the oracle's two-mode compressor's error, and a mode-11 block's indices are each the best of the 16
    for its endpoints; mode-11 lattice blocks are reproduced exactly, in mode 11."""
    bcf = _bcf()
    rng = np.random.default_rng(zlib.crc32(("c/" + "/".join(kinds)).encode()))
    res, levels = 32, 4
    tex = np.concatenate([(_mode11_level(rng, res >> l) if kinds[l % len(kinds)] == "mode11"
                           else _level_texels(rng, res >> l, kinds[l % len(kinds)])).reshape(-1)
                          for l in range(levels)])
    blocks, err, modes = bcf.compress_bc6h(torch.from_numpy(tex).cuda(), res, levels)
    blocks, err, modes = blocks.cpu().numpy().reshape(-1, 16), err.cpu().numpy(), modes.cpu().numpy()
    _, rerr, rmodes = oracle.compress_bc6h_texture(tex, res, levels)
    targets = _block_targets(tex, res, levels)
    for b in range(blocks.shape[0]):
        mode = oracle.bc6h_block_mode(blocks[b])
        assert mode == modes[b] and mode in (10, 11), (b, mode, modes[b])
        tgt = targets[b].astype(np.float64)
        dec = ((_values(blocks[b]) - tgt) ** 2).sum()
        assert err[b] == pytest.approx(dec, rel=1e-5, abs=1e-9), (b, err[b], dec)
        assert dec <= rerr[b] * (1 + 1e-5) + 1e-12, (b, dec, rerr[b], mode, rmodes[b])
        if mode == 11:
            e = _mode11_endpoints(blocks[b])
            for t in range(16):
                errs = [((oracle_mode11_value(e, i) - tgt[t]) ** 2).sum() for i in range(16)]
                got = ((_values(blocks[b])[t] - tgt[t]) ** 2).sum()
                assert got <= min(errs) * (1 + 1e-6) + 1e-12, (b, t)
    if "mode11" in kinds:  # the mode-11 lattice level is reproduced exactly, in mode 11
        lv = kinds.index("mode11")
        a = sum(((res >> l) // 4) ** 2 for l in range(lv))
        b = a + ((res >> lv) // 4) ** 2
        assert (modes[a:b] == 11).all() and not err[a:b].any()


def _mode11_endpoints(blk):
    """The two 10-bit endpoints (RGB) of a mode-11 block, read from its fields: bits 5..64, RGB of the first
    endpoint then of the second, 10 bits each."""
    bits = np.unpackbits(np.asarray(blk, np.uint8), bitorder="little")
    vals = [int(sum(int(bits[5 + 10 * j + i]) << i for i in range(10))) for j in range(6)]
    return np.array(vals).reshape(2, 3)


def oracle_mode11_value(e, i):
    """Value of index i between 10-bit endpoints e[0], e[1], through the format decoder (a block whose texel 0
    carries the index; mirrored when the anchor rule requires)."""
    raw = [int(v) for v in np.asarray(e).reshape(-1)] + [0] * 6
    ii = [int(i)] + [0] * 15
    if i >= 8:
        raw = raw[3:6] + raw[0:3] + [0] * 6
        ii = [15 - j for j in ii]
    return _values(oracle.bc6h_encode_fields(11, raw, 0, ii))[0]


def test_compressor_output_is_a_texture_the_decoder_takes():
    """The compressed blocks decode (bcf_decode_bc6h, every level) to values whose squared error against the
    input is the reported error."""
    bcf = _bcf()
    rng = np.random.default_rng(71)
    res, levels = 16, 3
    tex = _texture(rng, res, levels, ("smooth", "noise"))
    blocks, err, _ = bcf.compress_bc6h(torch.from_numpy(tex).cuda(), res, levels)
    off_b, off_t = 0, 0
    for lvl in range(levels):
        W = res >> lvl
        nb = (W // 4) ** 2
        dec = bcf.decode_bc6h(blocks[16 * off_b:16 * (off_b + nb)], W // 4, W // 4).cpu().numpy()
        vals = dec.view(np.float16).astype(np.float32).reshape(W, W, 3)
        src = tex[off_t:off_t + W * W * 3].reshape(W, W, 3)
        sq = ((vals - src) ** 2).reshape(W // 4, 4, W // 4, 4, 3).transpose(0, 2, 1, 3, 4).reshape(nb, 48)
        np.testing.assert_allclose(sq.astype(np.float64).sum(1), err[off_b:off_b + nb].cpu().numpy(), rtol=1e-5,
                                   atol=1e-9)
        off_b += nb
        off_t += W * W * 3
