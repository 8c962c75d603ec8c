// echo_batch_f64.cu -- batched-run kernels for double storage.
#include "echo_batch_kernels.cuh"

namespace echo {

template <>
const void *batch_stage_kernel<double>(int mk, bool mlp)
{
    if (mk == 1)
        return mlp ? (const void *)k_batch_stage<1, double, true, 4> : (const void *)k_batch_stage<1, double, false, 4>;
    return mlp ? (const void *)k_batch_stage<0, double, true, 4> : (const void *)k_batch_stage<0, double, false, 4>;
}

template <int MK>
static void phased(bool mlp, const RunDesc<double> *descs, const BatchPlan *planp, const BatchPlan &P, int nruns,
                   const Phys &ph, int guess, double dt, double cfl, cudaStream_t s)
{
    k_bphase_scalars<double><<<1, 32, 0, s>>>(descs, nruns, 0, dt, cfl);
    for (int st = 0; st < 3; ++st) {
        for (int p = PH_FILLF0; p <= PH_FILLF2; ++p)
            k_bphase_fill<double><<<(unsigned)P.ntiles[p], 128, 0, s>>>(descs, planp, p);
        if (mlp)
            k_bphase_c2p<MK, double, true><<<(unsigned)P.ntiles[PH_C2P], 128, MLP_BLOCK * sizeof(float), s>>>(
                descs, planp, ph, guess, st == 0 ? 1 : 0);
        else
            k_bphase_c2p<MK, double, false><<<(unsigned)P.ntiles[PH_C2P], 128, 0, s>>>(descs, planp, ph, guess,
                                                                                   st == 0 ? 1 : 0);
        if (st == 0)
            k_bphase_scalars<double><<<1, 32, 0, s>>>(descs, nruns, 1, dt, cfl);
        for (int p = PH_FILLP0; p <= PH_FILLP2; ++p)
            k_bphase_fill<double><<<(unsigned)P.ntiles[p], 128, 0, s>>>(descs, planp, p);
        k_bphase_faces<MK, double><<<(unsigned)P.ntiles[PH_FACES], 128, 0, s>>>(descs, planp, ph);
        k_bphase_emf<MK, double><<<(unsigned)P.ntiles[PH_EMF], 128, 0, s>>>(descs, planp);
        k_bphase_update<MK, double><<<(unsigned)P.ntiles[PH_UPDATE], 128, 0, s>>>(descs, planp, ph, st);
    }
}

template <>
void batch_enqueue_phased<double>(int mk, bool mlp, const void *descs, const BatchPlan *plan_dev, const BatchPlan &plan,
                              int nruns, const Phys &ph, int guess, double dt, double cfl, cudaStream_t s)
{
    const RunDesc<double> *d = static_cast<const RunDesc<double> *>(descs);
    if (mk == 1)
        phased<1>(mlp, d, plan_dev, plan, nruns, ph, guess, dt, cfl, s);
    else
        phased<0>(mlp, d, plan_dev, plan, nruns, ph, guess, dt, cfl, s);
}

}  // namespace echo
