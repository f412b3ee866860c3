"""Plain PyTorch fp32 (CPU) restatement of the refiner network, for the GPU parity tests.

Parameters follow the library's layout: per layer W[tap = 3 ky + kx][Cout][Cin] then
b[Cout]; layers 16 -> 32 -> 32 -> 32 -> 32 -> 16 (ReLU after the first four), output =
plain + channel 0 of the last layer.  `forward` rounds weights and hidden activations to
bf16 as the kernels store them (straight through for the gradient) and, for training, the
gradients the kernels store in bf16; everything else fp32.
"""
import numpy as np
import torch
import torch.nn.functional as F

CIN = (16, 32, 32, 32, 32)
COUT = (32, 32, 32, 32, 16)
NPARAM = sum(9 * ci * co + co for ci, co in zip(CIN, COUT))


def layers(params):
    """[(weight offset, W torch [co][ci][3][3], bias offset, b torch [co])]"""
    off, out = 0, []
    for ci, co in zip(CIN, COUT):
        w = torch.tensor(params[off:off + 9 * ci * co].reshape(3, 3, co, ci)).permute(2, 3, 0, 1)
        wo = off
        off += 9 * ci * co
        b = torch.tensor(params[off:off + co])
        out.append((wo, w.contiguous(), off, b))
        off += co
    assert off == len(params) == NPARAM
    return out


def bf(x):
    return x.to(torch.bfloat16).to(torch.float32)


class _GradToBf16(torch.autograd.Function):
    """Identity forward; the gradient is rounded to bf16 on the way back, as the kernels
    store the gradient of every layer's pre-activation (and of the output) in bf16."""

    @staticmethod
    def forward(ctx, x):
        return x.view_as(x)

    @staticmethod
    def backward(ctx, g):
        return bf(g)


def forward(params, x0, plain, gt=None, bf16_grads=True):
    """x0 [N][H][W][16] (fp32 holding bf16 values), plain/gt [N][H][W] fp32 numpy or torch.

    With bf16_grads the gradients of the pre-activations and of the output are rounded to
    bf16 on the way back, where the kernels store them.  Returns (out numpy [N][H][W],
    loss or None, grads numpy [NPARAM] or None)."""
    ls = layers(np.asarray(params, dtype=np.float32))
    ws, bs = [], []
    h = torch.as_tensor(np.asarray(x0, dtype=np.float32)).permute(0, 3, 1, 2)
    for l, (_, w, _, b) in enumerate(ls):
        wq = bf(w).requires_grad_(gt is not None)
        bq = b.clone().requires_grad_(gt is not None)
        ws.append(wq)
        bs.append(bq)
        z = F.conv2d(h, wq, bq, padding=1)
        if gt is not None and bf16_grads and l < len(ls) - 1:
            z = _GradToBf16.apply(z)
        if l < len(ls) - 1:
            r = torch.relu(z)
            h = r + (bf(r) - r).detach()
        else:
            out = z[:, 0] + torch.as_tensor(np.asarray(plain, dtype=np.float32))
    if gt is None:
        return out.detach().numpy(), None, None
    if bf16_grads:
        out = _GradToBf16.apply(out)
    loss = torch.mean((out - torch.as_tensor(np.asarray(gt, dtype=np.float32))) ** 2)
    loss.backward()
    g = np.zeros(NPARAM, dtype=np.float32)
    for (wo, w, bo, b), wq, bq in zip(ls, ws, bs):
        g[wo:wo + w.numel()] = wq.grad.permute(2, 3, 0, 1).reshape(-1).numpy()
        g[bo:bo + b.numel()] = bq.grad.numpy()
    return out.detach().numpy(), float(loss.detach()), g
