/* Polynomial coefficients of the FP64 oracle (design constants chosen by
 * the minimax fits in oracle/coeffs/; the CUDA sources carry the same
 * literals).  Constant term first. */
#ifndef ORACLE_COEFFS64_H
#define ORACLE_COEFFS64_H
#define EXP_U10_COEFFS 0x1.0000000000000p-1, 0x1.555555555555bp-3, 0x1.5555555555503p-5, 0x1.111111110ec3fp-7, 0x1.6c16c16c305dap-10, 0x1.a01a01b38a1ccp-13, 0x1.a01a01364ed77p-16, 0x1.71ddf0027528ep-19, 0x1.27e5b4917ffe5p-22, 0x1.af6c1dcd03fd7p-26, 0x1.1e3d09ab8b9a5p-29
#define EXP_U35_COEFFS 0x1.ffffffffffed1p-2, 0x1.5555555550776p-3, 0x1.5555555589411p-5, 0x1.11111125c3b1dp-7, 0x1.6c16c0c7b3762p-10, 0x1.a0198d1cfb5cfp-13, 0x1.a01b7d10e56f2p-16, 0x1.72e95f1b1c6d2p-19, 0x1.27076dd8a5103p-22
#define LOG_U10_COEFFS 0x1.555555555554fp-4, 0x1.999999999c179p-7, 0x1.24924921e457cp-9, 0x1.c71c748fb0e5ep-12, 0x1.745c4adfd4929p-14, 0x1.3b35c02f141cfp-16, 0x1.0dcba14fc06c7p-18, 0x1.1b8139759f314p-20
#define LOG_U35_COEFFS 0x1.5555555555775p-4, 0x1.99999998f0e71p-7, 0x1.249249b213a2dp-9, 0x1.c71c01680d46ap-12, 0x1.7474e2e4fcac3p-14, 0x1.3852c703d6843p-16, 0x1.3abef8cc48463p-18
#define POWLOG_C1H 0x1.5555555555555p-4
#define POWLOG_C1L 0x1.54855a03b34d8p-58
#define POWLOG_COEFFS 0x1.999999999999cp-7, 0x1.2492492492062p-9, 0x1.c71c71c78a1b0p-12, 0x1.745d171399b86p-14, 0x1.3b13bf3c5b892p-16, 0x1.110e98ef52765p-18, 0x1.e26f3be0efb86p-21, 0x1.a57c235e7b51bp-23, 0x1.e37c78d194e20p-25
#define POWEXP_COEFFS 0x1.555555555555ap-3, 0x1.5555555555498p-5, 0x1.111111110f0acp-7, 0x1.6c16c16c4d9f3p-10, 0x1.a01a01b2b4f71p-13, 0x1.a01a010b94555p-16, 0x1.71ddf039a6182p-19, 0x1.27e54bd4df84bp-22, 0x1.af6e560a2694ap-26, 0x1.1fda157dfad50p-29
#define ASIN_U10_COEFFS 0x1.5555555555577p-3, 0x1.333333332e131p-4, 0x1.6db6db7212680p-5, 0x1.f1c71a94f2d61p-6, 0x1.6e8bdee04467bp-6, 0x1.1c49f05c614d5p-6, 0x1.ca1f8d8013edbp-7, 0x1.75858907d1626p-7, 0x1.613c905725fb1p-7, 0x1.e5f54ce7fcfd8p-9, 0x1.639c82c0224b6p-6, -0x1.57fd8f93ea512p-6, 0x1.0b46c1e48a247p-5
#define ASIN_U35_COEFFS 0x1.5555555556cffp-3, 0x1.3333333091736p-4, 0x1.6db6dd0ddeac7p-5, 0x1.f1c69c91bed2cp-6, 0x1.6e97027d9cfafp-6, 0x1.1baccf082d699p-6, 0x1.d54ed312773eep-7, 0x1.336c9afab279ep-7, 0x1.2b0852e644fbbp-6, -0x1.7f68404d9c380p-7, 0x1.023493a75851bp-5
#define ATAN_U10_C1H -0x1.555555555554dp-2
#define ATAN_U10_C1L 0x1.f6f1c78b4061fp-57
#define ATAN_U10_COEFFS 0x1.9999999998c27p-3, -0x1.2492492456a9cp-3, 0x1.c71c71b628925p-4, -0x1.745d15d02799cp-4, 0x1.3b139bce356edp-4, -0x1.1110326711fe3p-4, 0x1.e1d487be7157ap-5, -0x1.aeda6036339c0p-5, 0x1.84b4dcab75621p-5, -0x1.5f276ea2a952dp-5, 0x1.3911a513777bbp-5, -0x1.0cba41b2fdaedp-5, 0x1.ad1808a727ccep-6, -0x1.31f10ec96d5a7p-6, 0x1.75115934da341p-7, -0x1.73826f657b4aap-8, 0x1.1e67b2bdce61dp-9, -0x1.3de0d575d18fdp-11, 0x1.c1459ac17e788p-14, -0x1.2e664c7ca4205p-17
#define ATAN_U35_COEFFS -0x1.555555555544cp-2, 0x1.999999998410ep-3, -0x1.2492491fa20b6p-3, 0x1.c71c709e18536p-4, -0x1.745d0230ed218p-4, 0x1.3b12b2e80c939p-4, -0x1.11089cfe49ae0p-4, 0x1.e1781718de794p-5, -0x1.ad32ba2f14c5ep-5, 0x1.7ee3f6bdf7ae1p-5, -0x1.4f4524eb17978p-5, 0x1.1715e3114eceep-5, -0x1.a726c401b7411p-6, 0x1.162c5d3e40d3ep-6, -0x1.2cf7a264b90d9p-7, 0x1.f96d516ef2061p-9, -0x1.312abcc54c86dp-10, 0x1.d3bc387104c94p-13, -0x1.53e7168f3586cp-16
#define CBRT_COEFFS 0x1.bf45ec441bd23p-1, -0x1.8d93481324a0ap-3, 0x1.6176914abb262p-4, -0x1.6ea83723fc3a3p-5, 0x1.925bc75c45e3cp-6, -0x1.cda96200ffa66p-7, 0x1.5223d83416936p-7, -0x1.a6ef2b72239f2p-8
#define EXPM1_U35_COEFFS 0x1.0000000000005p-1, 0x1.5555555555539p-3, 0x1.555555555228ep-5, 0x1.1111111119010p-7, 0x1.6c16c17ee7257p-10, 0x1.a01a0174fb45ep-13, 0x1.a019a74a758d7p-16, 0x1.71de882490dc7p-19, 0x1.28a2068fa4cf1p-22, 0x1.ae6bacbadab12p-26
/* erf: erf(x)/x = C0 + t (C1 + t P(t)) on t = x^2 in [0, 1]; erfc: F(x) = erfc(x) e^(x^2)
 * on [1,2), [2,4), [4,8) about the midpoints and G(w) = sqrt(pi) x F(x), w = 1/x^2 <= 1/64;
 * HEAD = c0 (hi, lo), c1 (hi, lo) */
#define ERF_A_HEAD 0x1.20dd750429b6dp+0, 0x1.18308016146fep-56, -0x1.812746b0379e6p-2, 0x1.dd80e959672c6p-58
#define ERF_A_COEFFS 0x1.ce2f21a042b20p-4, -0x1.b82ce31284967p-6, 0x1.565bcd0daf845p-8, -0x1.c02db3d8c8f93p-11, 0x1.f9a3219c76949p-14, -0x1.f4d1ded722b03p-17, 0x1.b9deec50ab26ap-20, -0x1.5f1d06eacf4c6p-23, 0x1.f7a1f36ad5781p-27, -0x1.3863e3c35d413p-30, 0x1.0566538cb8283p-34
#define ERFC_F0_HEAD 0x1.494daffa2ad68p-2, 0x1.39bdf0f0798c4p-56, -0x1.4f1988444caf7p-3, 0x1.24ac537655c12p-57
#define ERFC_F0_COEFFS 0x1.37ea271bc54bdp-4, -0x1.0dc51d2941e6dp-5, 0x1.b65944f34f7adp-7, -0x1.513ed7600d1c0p-8, 0x1.ee705e736464dp-10, -0x1.5b0abfe65a32dp-11, 0x1.d4509d0d417b9p-13, -0x1.30c0ec743bcedp-14, 0x1.7f997923557c4p-16, -0x1.d4157188ae920p-18, 0x1.156c936a3105dp-19, -0x1.4004eff6f7f58p-21, 0x1.67cf5f0988c05p-23, -0x1.8adc1a9fe6189p-25, 0x1.a779871f4a7bdp-27, -0x1.bc5770d3295a2p-29, 0x1.c8a6eada5b280p-31, -0x1.cbfeb0383b565p-33, 0x1.c520022695974p-35, -0x1.b81dd79ebf9adp-37, 0x1.c82b760607022p-39, -0x1.a70fd6017ce87p-41
#define ERFC_F1_HEAD 0x1.6e9827d229d2dp-3, -0x1.90756fe6b9db3p-58, -0x1.bd6ae4d14b16fp-5, 0x1.8d8b238907b15p-61
#define ERFC_F1_COEFFS 0x1.043fe1a98c0cdp-6, -0x1.259061ba85692p-8, 0x1.409cc2ed3fefbp-10, -0x1.53dec9d089553p-12, 0x1.5e739304850bcp-14, -0x1.6025103c1981bp-16, 0x1.595f1b5dbff18p-18, -0x1.4b14628647c09p-20, 0x1.369904b947a56p-22, -0x1.1d791455a0f11p-24, 0x1.01508df8e0a1fp-26, -0x1.c752068f0a96ep-29, 0x1.8bbf3f6db12c5p-31, -0x1.522804d7a7020p-33, 0x1.1c3dc4fa8a305p-35, -0x1.d66d6369f7643p-38, 0x1.8003b981c62cdp-40, -0x1.3453718d4c0bfp-42, 0x1.dbc8fa69f1588p-45, -0x1.7551e98792b95p-47, 0x1.6ca3dddd58940p-49, -0x1.10f3c57b6b0d7p-51
#define ERFC_F2_HEAD 0x1.7c0348489d721p-4, 0x1.ca79ab435b660p-58, -0x1.ed7f66d9d09fep-7, 0x1.3b520acfa96f3p-62
#define ERFC_F2_COEFFS 0x1.3c7764a81f462p-9, -0x1.9106a7cd79e3bp-12, 0x1.f64cd9c07b5c5p-15, -0x1.370d0641775e4p-17, 0x1.7d0e03edb73e5p-20, -0x1.cde4cecce654ep-23, 0x1.1513469d8602cp-25, -0x1.491bb0ca940c5p-28, 0x1.83201ae0eb1dcp-31, -0x1.c312ca4fcf13cp-34, 0x1.045ff3e648ff3p-36, -0x1.29e5d7aaf7613p-39, 0x1.51dbcb9512727p-42, -0x1.7be13c8006386p-45, 0x1.a72a1d41d3c2ap-48, -0x1.d40a279e38d1dp-51, 0x1.040a46c482170p-53, -0x1.1a97bd1e37a50p-56, 0x1.0dfc0cce80407p-59, -0x1.24502b98063a1p-62, 0x1.0709dd4f990c4p-64, -0x1.11b59748cdbf2p-67
#define ERFC_G_HEAD 0x1.0000000000000p+0, -0x1.38b4a1f7dc331p-66, -0x1.ffffffffffffbp-2, -0x1.449ed132ba430p-56
#define ERFC_G_COEFFS 0x1.7ffffffffe83fp-1, -0x1.dffffffd0f32bp+0, 0x1.a3fffe80c9ac6p+2, -0x1.d87f8dc75c4bdp+4, 0x1.44cd52e365bc6p+7, -0x1.0749c46c91cccp+10, 0x1.e1ba8d8295a72p+12, -0x1.b7be9d06eea96p+15, 0x1.142dd87ba7a2cp+18
/* lgamma: lgamma(2 + e) = e (c1 + e (c2 + e P)) on [-0.25, 0.5]; lgamma(1.5 + u) = c0 + u (c1 + u (c2 + u P))
 * on [-0.25, 0.25]; Stirling correction x S(x) in w = 1/x^2 on [0, 1/64]; sin(pi s) = s (pi + t (c1 + t P)) */
#define LGAMMA_R2_HEAD 0x1.b0ee6072093cep-2, 0x1.6c58518ef209cp-58, 0x1.4a34cc4a60fa6p-2, 0x1.1b98b7d24eb82p-56
#define LGAMMA_R2_COEFFS -0x1.13e001a557606p-4, 0x1.51322ac7d846dp-6, -0x1.e404fc218fc23p-8, 0x1.7add6eadbd405p-9, -0x1.38ac5c2b8a199p-10, 0x1.0b36af7f23772p-11, -0x1.d3fd4cdaf22e0p-13, 0x1.a127b9082ca84p-14, -0x1.78de521792e56p-15, 0x1.580b6a9b7953fp-16, -0x1.3cb65d569461dp-17, 0x1.25e70a4f871bep-18, -0x1.139ba270fa662p-19, 0x1.ffad5d0754437p-21, -0x1.99a8f419f8596p-22, 0x1.7da6d390ec3f8p-24
#define LGAMMA_M_HEAD -0x1.eeb95b094c191p-4, -0x1.34022180247c2p-58, 0x1.2aed059bd608ap-5, 0x1.7e1a96f7c7ed0p-63, 0x1.de9e64df22ef3p-2, -0x1.b1d5ff59dcc8fp-56
#define LGAMMA_M_COEFFS -0x1.1ae55b180726bp-3, 0x1.e0f840dad650ap-5, -0x1.da59d5374aed9p-6, 0x1.f9ca39da28ed7p-7, -0x1.1a8ba4f054ba6p-7, 0x1.456f1b2745dc9p-8, -0x1.7edb81cde7f7cp-9, 0x1.c973218d36f11p-10, -0x1.148a003bbd58dp-10, 0x1.51884c3b797c0p-11, -0x1.9f11b5ad1c5d2p-12, 0x1.fea4040bd8d69p-13, -0x1.3d5aec9602328p-13, 0x1.bf0b984ee3abdp-14, -0x1.1a86a63641821p-14
#define LGAMMA_ST_COEFFS 0x1.5555555555555p-4, -0x1.6c16c16c16c16p-9, 0x1.a01a01a0196bap-11, -0x1.381381362b216p-11, 0x1.b951df87db260p-11, -0x1.f6a98a1bab42ap-10, 0x1.a3e150e3f70bdp-8, -0x1.dee553034d0abp-6, 0x1.490abb645435cp-3, -0x1.7031193624fc5p-1
#define SINPI_HEAD -0x1.4abbce625be53p+2, 0x1.05511c684d1cbp-52
#define SINPI_COEFFS 0x1.466bc6775aae2p+1, -0x1.32d2cce62bddep-1, 0x1.50783487f6d9cp-4, -0x1.e3074fec25b1dp-8, 0x1.e8f4422d6f029p-12, -0x1.6fb6226ceb4fdp-16, 0x1.b1dd7b5e6be80p-21, -0x1.5249d9e04752dp-24, 0x1.46d5e635ea9dep-23, -0x1.f9b2ef7ed3d1ep-23, 0x1.563183599af6cp-23
/* C99 set: sin(pi s) = s (c0 + t (c1 + t P(t))) and cos(pi s) = 1 + t (c0 + t P(t)),
 * t = s^2 in [0, 1/16]; HEAD = the DD leading coefficients (oracle/coeffs/fit_c99.py) */
#define C99_SINPI_HEAD 0x1.921fb54442d18p+1, 0x1.1a5ee6df61731p-53, -0x1.4abbce625be53p+2, 0x1.1317e21cffea3p-52
#define C99_SINPI_COEFFS 0x1.466bc6775aad9p+1, -0x1.32d2cce62ac1bp-1, 0x1.50783485cd9dep-4, -0x1.e3074b54cb043p-8, 0x1.e8eed5bfbbb87p-12, -0x1.6c5d06da75ea5p-16
#define C99_COSPI_HEAD -0x1.3bd3cc9be45dep+2, -0x1.692b254f96cb6p-52
#define C99_COSPI_COEFFS 0x1.03c1f081b5ac4p+2, -0x1.55d3c7e3cc16cp+0, 0x1.e1f5068965fb7p-3, -0x1.a6d1f30fc0185p-6, 0x1.f9d42dc364f31p-10, -0x1.b7598d34a382dp-14, 0x1.41f35eddaaed2p-18
#endif
