"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np
import torch

TOL_IMG_F32 = 1e-5      # absolute, FP32 path image vs the FP64 oracle
TOL_IMG_BF16 = 2e-3     # absolute, BF16-field image vs the FP64 oracle
TOL_GRAD_F32 = 1e-3     # relative L2, FP32 path gradients
TOL_GRAD_BF16 = 2e-2    # relative L2, BF16 path gradients
# FP32 path with "trained-like" tables (U(+-0.5) instead of the configs'
# U(+-1e-4)): FP32 hash coordinates resolve the finest level (resolution
# 7006) only to ~7006 * 2^-24 ~ 4e-4 of a cell, so features move by up to
# ~4e-4 x the corner spread (~1); through the decoders this bounds the image
# error near 1e-4.
TOL_IMG_F32_TRAINED = 1e-4
TOL_Q_F32 = 2e-6        # field-query outputs, configs' initialisation
TOL_Q_F32_TRAINED = 2e-4


def rect_flip_tiles(rect_a, rect_b, tiles_x):
    """Tiles covered by exactly one of two rectangle lists (decisions that
    differ because the FP32 inputs of the two sides differ)."""
    import numpy as np
    out = set()
    diff = np.nonzero((rect_a != rect_b).any(1))[0]
    for i in diff:
        ta = {(y, x) for y in range(rect_a[i, 1], rect_a[i, 3]) for x in range(rect_a[i, 0], rect_a[i, 2])}
        tb = {(y, x) for y in range(rect_b[i, 1], rect_b[i, 3]) for x in range(rect_b[i, 0], rect_b[i, 2])}
        out |= {y * tiles_x + x for (y, x) in ta ^ tb}
    return out, len(diff)


def tile_mask(tiles, W, H, tile=16):
    import numpy as np
    m = np.zeros((H, W), bool)
    TX = (W + tile - 1) // tile
    for t in tiles:
        y, x = divmod(t, TX)
        m[y * tile:(y + 1) * tile, x * tile:(x + 1) * tile] = True
    return m


def np_(t):
    return t.detach().float().cpu().numpy() if t.dtype in (torch.bfloat16, torch.float16) else \
        t.detach().cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def cuda_f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def cuda_i32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).cuda()
