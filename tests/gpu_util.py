"""Helpers shared by the GPU parity tests (not collected as tests)."""
import numpy as np
import torch

TOL_IMG_F32 = 1e-5      # absolute, FP32 path image vs the FP64 oracle
TOL_IMG_BF16 = 2e-3     # absolute, BF16-field image vs the FP64 oracle
TOL_GRAD_F32 = 1e-3     # relative L2, FP32 path gradients
TOL_GRAD_BF16 = 2e-2    # relative L2, BF16 path gradients
# FP32 path with "trained-like" tables (U(+-0.5) instead of the configs'
# U(+-1e-4)). FP32 hash coordinates resolve the finest level (resolution
# 7006) to ~7006 * 2^-24 ~ 4e-4 of a cell (Gaussians) and, for background
# points on the radius-100 sphere, to ~1e-3 of a cell (the ray/sphere hit is
# ~1e-7 relative); features then move by that fraction of the corner spread
# (up to 1), which the decoders carry to the outputs. Bounds used here:
TOL_IMG_F32_TRAINED = 2e-3
TOL_GRAD_F32_TRAINED = 1e-2
TOL_Q_F32 = 2e-6        # field-query outputs, configs' initialisation
TOL_Q_F32_TRAINED = 2e-4
# BF16 decoders against the oracle that takes its ReLU branches in the
# kernel's precision (oracle.replay_relu(fields, "bf16")): a row or pixel is
# left out of a gradient comparison only when one of its hidden
# pre-activations lies within this relative margin of zero in the replay.
# What is left to flip a branch is the FP32 hash coordinate of the kernel
# (features off by ~1e-3 of a bfloat16 step, which moves a pre-activation by
# ~1e-4 of its magnitude at most) and FP32 accumulation (~1e-7).
RELU_REPLAY_MARGIN_BF16 = 2e-4


def np_(t):
    return t.detach().float().cpu().numpy() if t.dtype in (torch.bfloat16, torch.float16) else \
        t.detach().cpu().numpy()


def rel_l2(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    den = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (den if den > 0 else 1.0)


def psnr(a, b):
    """PSNR in dB of image a against image b (values clipped to [0, 1])."""
    a = np.clip(np.asarray(a, np.float64), 0.0, 1.0)
    b = np.clip(np.asarray(b, np.float64), 0.0, 1.0)
    return float(-10.0 * np.log10(np.mean((a - b) ** 2)))


def cuda_f32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def cuda_i32(a):
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.int32)).cuda()
