"""GB300-native occupancy-grid ray marching and packed differentiable volume rendering.

The method is NerfAcc's (arXiv 2210.04847): ray marching that skips empty space
with a binary occupancy grid (Sec. 2.1), pruning by early stopping on
transmittance and by an opacity threshold (Sec. 2.1), and differentiable
rendering of packed samples with the quadrature of Eq. 1 (Sec. 2.2).
"""
__version__ = "0.1.0"
