"""FP64 CPU oracle for damped parallel EP with an anisotropic l1-TV prior.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
restatement of the method of Yao, McLaughlin and Altmann, "Fast Scalable Image
Restoration using Total Variation Priors and Expectation Propagation"
(arXiv:2110.01585), used to check the CUDA library.  Only the test-suite, the
smoke check of ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may
import it.  The CUDA product path never imports, links or calls anything here,
and nothing here imports the CUDA path.

Modules
-------
tilted     Moments of the tilted law of one edge difference (Sec. III-C,
           Eq. marginal_tilted_un) for the three priors of Sec. II-B: the
           Laplace factor of l1-TV (the paper omits the closed forms; they are
           derived in the module docstring) and the two-Gaussian factors of
           MoG2-TV and BG-TV.
partition  The four matchings V1..V4 of the 4-neighbour graph (Sec. II-B,
           Eq. prior1 and the caption of Fig. 1).
operators  The degradation operators H (identity, periodic convolution, dense
           matrix), written from their definitions (Sec. II-A).
ep         Algorithm 1 (EP sweep) and Algorithm 2 (EP-EM), with the site
           updates Eq. update_q0_x / Eq. update_qk_x, the projection of the
           edge moments onto the two pixels, the recombination Eq. Q_x_final,
           the variance cap and damping of Sec. III-C.
cnn        The convolutional network of the learned warm start (not in the
           paper): circular 3x3 convolutions, ReLU, their gradients, the Adam
           step and the training loss.

Every floating-point quantity is float64.
"""
